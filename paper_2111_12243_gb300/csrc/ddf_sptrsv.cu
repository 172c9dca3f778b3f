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
#include <algorithm>

#include "ddf_internal.cuh"

namespace {


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
// rows, v lanes per row).  Warp gw of W runs units gw, gw + W, gw + 2W, ...
// and software-pipelines them: what a unit needs before its dependencies can
// be read comes through three dependent loads (the unit record and its first
// position; then the codelet descriptor, the row, its value extent and
// 1 / L_ii; then the values, the columns and b), so while the warp waits on
// unit k's dependencies it already issues the third level of loads for unit
// k+1, the second for unit k+2 and the first for unit k+3.  When unit k's
// dependencies are ready, only their flag hop is left on the critical path.
constexpr int SOLVE_SMAX = DDF_SOLVE_PTS;   // points per lane held in registers (rows of up to SMAX v points)

struct SolveL1 {                // level 1: unit record
    int32_t cod, i0b, i0e, v, qb;
};
template <typename TX>
struct SolveL2 {                // level 2: descriptor fields, row, value extent, 1 / L_ii
    int32_t v, li, q, act;
    int32_t cq0, ctype, ch0, cdelta, csigma, csref;
    int32_t r, s0, s1;
    TX di;
};
template <typename TV, typename TX>
struct SolveL3 {                // level 3: values, columns, b
    int32_t v, li, act, r, L, kb, hb, type, sigma, sref, h0, joff;
    TX di, bv;
    TV vv[SOLVE_SMAX];
    int32_t jraw[SOLVE_SMAX];
};

__device__ __forceinline__ void solve_ld1(const dunit* __restrict__ units, const int32_t* __restrict__ unit_q,
                                          int64_t u, int64_t nunits, SolveL1& a) {
    if (u < nunits) {
        const int4 t = __ldg(reinterpret_cast<const int4*>(units + u));
        a.cod = t.x;
        a.i0b = t.y;
        a.i0e = t.z;
        a.v = t.w;
        a.qb = __ldg(unit_q + u);
    } else {
        a.cod = -1;
        a.i0b = a.i0e = a.qb = 0;
        a.v = 32;
    }
}

template <typename TX>
__device__ __forceinline__ void solve_ld2(const SolveL1& a, int lane, const dcod* __restrict__ cod,
                                          const int32_t* __restrict__ seq, const int32_t* __restrict__ st,
                                          const TX* __restrict__ dinv, SolveL2<TX>& c) {
    const int lg = __ffs(a.v) - 1;
    const int sub = lane >> lg;
    c.v = a.v;
    c.li = lane & (a.v - 1);
    c.act = a.cod >= 0 && a.i0b + sub < a.i0e;
    c.q = a.qb + sub;
    c.cq0 = c.ctype = c.ch0 = c.cdelta = c.csigma = c.csref = 0;
    c.r = c.s0 = c.s1 = 0;
    c.di = 0;
    if (a.cod >= 0) {
        const dcod* C = cod + a.cod;
        c.cq0 = __ldg(&C->q0);
        c.ctype = __ldg(&C->type);
        c.ch0 = __ldg(&C->h0);
        c.cdelta = __ldg(&C->delta);
        c.csigma = __ldg(&C->sigma);
        c.csref = __ldg(&C->sref);
    }
    if (c.act) {
        c.r = __ldg(seq + c.q);
        c.s0 = __ldg(st + c.q);
        c.s1 = __ldg(st + c.q + 1);
        c.di = __ldg(dinv + c.q);
    }
}

template <typename TV, typename TX>
__device__ __forceinline__ void solve_ld3(const SolveL2<TX>& c, const int32_t* __restrict__ col,
                                          const TV* __restrict__ val, const TX* __restrict__ b,
                                          SolveL3<TV, TX>& d) {
    d.v = c.v;
    d.li = c.li;
    d.act = c.act;
    d.r = c.r;
    d.di = c.di;
    d.type = c.ctype;
    d.sigma = c.csigma;
    d.sref = c.csref;
    d.h0 = c.ch0;
    d.kb = c.s0;
    d.L = c.act ? c.s1 - c.s0 : 0;
    d.hb = c.ch0 + c.cdelta * (c.q - c.cq0);
    d.joff = c.ctype == DDF_PSC1 ? d.hb - c.ch0 : 0;
    d.bv = c.act ? __ldg(b + c.r) : (TX)0;
#pragma unroll
    for (int k = 0; k < SOLVE_SMAX; ++k) {
        const int32_t i1 = d.li + k * d.v;
        d.vv[k] = (TV)0;
        d.jraw[k] = 0;
        if (i1 < d.L) {
            d.vv[k] = __ldg(val + d.kb + i1);
            d.jraw[k] = d.type == DDF_BLAS   ? d.hb + d.sigma * i1
                        : d.type == DDF_PSC1 ? __ldg(col + d.sref + i1)
                                             : __ldg(col + d.kb + i1);
        }
    }
}

template <typename TV, typename TX>
__global__ void __launch_bounds__(DDF_CTA_THREADS, DDF_SOLVE_CTAS_PER_SM)
k_sptrsv(const dcod* __restrict__ cod, const dunit* __restrict__ units, const int32_t* __restrict__ unit_q,
         int64_t nunits, const int32_t* __restrict__ seq, const int32_t* __restrict__ st,
         const int32_t* __restrict__ col, const TV* __restrict__ val, const TX* __restrict__ dinv,
         const TX* __restrict__ b, TX* x, uint32_t* ticket, int32_t* status, int64_t cap_ns) {
    using B = XBits<TX>;
    uint32_t* abort_flag = ticket + 1;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t u0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u0 >= nunits) return;   // warp-uniform
    // prologue: unit 0 to level 3, unit 1 to level 2, unit 2 to level 1
    SolveL1 t0, t1, t2;
    solve_ld1(units, unit_q, u0, nunits, t0);
    solve_ld1(units, unit_q, u0 + nw, nunits, t1);
    solve_ld1(units, unit_q, u0 + 2 * nw, nunits, t2);
    SolveL2<TX> c0, c1;
    solve_ld2<TX>(t0, lane, cod, seq, st, dinv, c0);
    solve_ld2<TX>(t1, lane, cod, seq, st, dinv, c1);
    SolveL3<TV, TX> cur;
    solve_ld3<TV, TX>(c0, col, val, b, cur);
    for (int64_t u = u0; u < nunits; u += nw) {
        // this unit's dependencies first
        typename B::U xv[SOLVE_SMAX];
#pragma unroll
        for (int k = 0; k < SOLVE_SMAX; ++k) {
            const int32_t i1 = cur.li + k * cur.v;
            xv[k] = i1 < cur.L ? B::ld(x + cur.jraw[k] + cur.joff) : (typename B::U)0;
        }
        // then the next units' loads, which land while this unit waits
        SolveL3<TV, TX> nxt;
        solve_ld3<TV, TX>(c1, col, val, b, nxt);
        SolveL2<TX> c2;
        solve_ld2<TX>(t2, lane, cod, seq, st, dinv, c2);
        SolveL1 t3;
        solve_ld1(units, unit_q, u + 3 * nw, nunits, t3);
        // While some dependencies held in registers are not ready, every lane
        // re-reads its own missing values, so one round trip checks all of
        // the warp's late dependencies at once; the next round is issued as
        // soon as the last returns (a pause between rounds measured slower).
        // The wait is bounded: every 16 rounds the warp checks the abort flag
        // and the time since it started waiting, and past cap_ns it latches
        // DDF_ERR_TIMEOUT.
        uint64_t tw = 0;
        uint32_t rounds = 0;
        while (true) {
            bool miss = false;
#pragma unroll
            for (int k = 0; k < SOLVE_SMAX; ++k) miss |= (cur.li + k * cur.v < cur.L) && xv[k] == B::SENT;
            if (!__any_sync(0xffffffffu, miss)) break;
            if (rounds == 0) tw = ddf_globaltimer();
            ++rounds;
            bool stop = false;
            if ((rounds & 15u) == 0) {
                const bool late = __any_sync(0xffffffffu, (int64_t)(ddf_globaltimer() - tw) > cap_ns);
                if (late && lane == 0) {
                    ddf_set_status(status, DDF_ERR_TIMEOUT);
                    atomicExch(abort_flag, 1u);
                }
                stop = late || __any_sync(0xffffffffu, ddf_ld_relaxed_s32(abort_flag) != 0);
            }
#pragma unroll
            for (int k = 0; k < SOLVE_SMAX; ++k)
                if ((cur.li + k * cur.v < cur.L) && xv[k] == B::SENT)
                    xv[k] = stop ? B::CANON : B::ld(x + cur.jraw[k] + cur.joff);
        }
        TX acc = 0;
        if (cur.act) {
#pragma unroll
            for (int k = 0; k < SOLVE_SMAX; ++k)
                if (cur.li + k * cur.v < cur.L) acc += ddf_cvt<TX>(cur.vv[k]) * B::val(xv[k]);
            // rows longer than SOLVE_SMAX * v points: the rest one by one
            for (int32_t i1 = cur.li + SOLVE_SMAX * cur.v; i1 < cur.L; i1 += cur.v) {
                const int32_t j = cur.type == DDF_BLAS   ? cur.hb + cur.sigma * i1
                                  : cur.type == DDF_PSC1 ? cur.hb + (col[cur.sref + i1] - cur.h0)
                                                         : col[cur.kb + i1];
                acc += ddf_cvt<TX>(val[cur.kb + i1]) * dep<TX>(x, j, status, abort_flag, cap_ns);
            }
        }
        for (int o = cur.v >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (cur.act && cur.li == 0) {
            TX xr = (cur.bv - acc) * cur.di;
            typename B::U bits = B::bits(xr);
            if (bits == B::SENT) bits = B::CANON;
            B::st(x + cur.r, bits);
        }
        cur = nxt;
        c1 = c2;
        t2 = t3;
    }
}

// ---------------------------------------------------------------------------
// Coarsened solve (plans with coarsen_rows = R > 0).  The partitions of a
// block of R consecutive rows are that block's level sets, so one CTA runs a
// whole block: the block's x lives in shared memory (xs), a dependency inside
// the block costs a shared-memory read behind a CTA-local barrier instead of
// a flag hop through L2, and only columns before the block's first row (the
// "external" prefix of a row, esplit[q] points) are read from other blocks
// through the x-as-flag protocol of the plain solve.
//
// The inspector cut every partition into chunks (at most DDF_BLK_ROWS_CAP rows
// and DDF_BLK_ENT_CAP points, positions consecutive), so a chunk's values and
// columns are one contiguous range of the plan's arrays.  Warp roles:
//   producers (BLK_PROD warps, one staging slot each): chunk k of the block
//     goes to producer k mod BLK_PROD.  It stages the chunk's values (and, for
//     chunks with PSC II rows, columns) into its slot with bulk copies (TMA,
//     completion on an mbarrier), reads each row's codelet, sets
//     xs[r - base] = b[r] - (external sum), rewrites each in-block column as
//     an offset into xs, and publishes the chunk.
//   chain (BLK_CHAIN warps): chunks in order; each row subtracts its in-block
//     points (all operands in shared memory), scales by 1 / L_ii, stores x in
//     xs and in global x; a named barrier among the chain warps ends a chunk.
// A producer reuses its slot only after the chain has finished the slot's
// previous chunk.  Blocks come from a ticket in increasing order and a block
// reads only rows of earlier blocks, which hold a ticket and run, so every
// wait ends; each is bounded by spin_cap_ns like those of the plain solve.
// ---------------------------------------------------------------------------
constexpr int BLK_CHAIN = DDF_BLK_CHAIN_LANES / 32;
constexpr int BLK_PROD_MAX = 12;                // producer warps (= staging slots), at most
constexpr int BLK_PB = DDF_BLK_PROD_PER_LANE;   // external points per producer lane per batch

__host__ __device__ constexpr int round16(int b) { return (b + 15) & ~15; }

// Byte layout of one staging slot: the chunk's values and columns (bulk
// copies, up to 15 bytes of alignment slack at each end), then per row its
// xs offset, value start, length, external count, and 1 / L_ii.
template <typename TV, typename TX>
struct SlotLayout {
    static constexpr int VAL = round16(DDF_BLK_ENT_CAP * (int)sizeof(TV) + 32);
    static constexpr int COL = round16(DDF_BLK_ENT_CAP * 4 + 32);
    static constexpr int META = DDF_BLK_ROWS_CAP * 16;            // int4 per row
    static constexpr int DINV = round16(DDF_BLK_ROWS_CAP * (int)sizeof(TX));
    static constexpr int BYTES = VAL + COL + META + DINV;
};

struct BlkShared {
    unsigned long long bar[BLK_PROD_MAX];   // one mbarrier per slot
    int32_t blk;
    int32_t chain_done;                     // chunks of the block finished by the chain
    int32_t ext_done[BLK_PROD_MAX];         // chunks finished by each producer
    int32_t crows[BLK_PROD_MAX];            // rows of the slot's current chunk
    int32_t cmeta[BLK_PROD_MAX];            // chunk_meta of the slot's current chunk
    int32_t dv[BLK_PROD_MAX], dc[BLK_PROD_MAX];   // element shift of the staged ranges
    int32_t e0[BLK_PROD_MAX];               // first value index of the chunk
    double red[BLK_CHAIN];                  // direct rows: per-warp partial sums
};

__device__ __forceinline__ int32_t ld_vol(const int32_t* p) { return *(const volatile int32_t*)p; }
__device__ __forceinline__ void st_vol(int32_t* p, int32_t v) { *(volatile int32_t*)p = v; }
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for a slot's staging to land.  The copies read this GPU's own
// memory and always complete; should the cap still run out the status is
// latched and the wait goes on for one more cap, so that no copy is left in
// flight when the kernel ends.
__device__ __noinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, int32_t* status,
                                       uint32_t* abort_flag, int64_t cap_ns) {
    uint64_t t0 = ddf_globaltimer();
    bool late = false;
    while (!mbar_try_wait(bar, parity)) {
        if ((int64_t)(ddf_globaltimer() - t0) > cap_ns) {
            if (late) return false;
            late = true;
            ddf_set_status(status, DDF_ERR_TIMEOUT);
            atomicExch(abort_flag, 1u);
            t0 = ddf_globaltimer();
        }
    }
    return true;
}

// Bounded wait until a shared counter reaches `need`.  Returns false when it
// gave up (this call's abort flag is set, or the cap ran out): the data the
// counter guards must then not be read.
__device__ __noinline__ bool wait_count(const int32_t* c, int32_t need, int32_t* status, uint32_t* abort_flag,
                                        int64_t cap_ns) {
    uint64_t t0 = ddf_globaltimer();
    uint32_t it = 0;
    while (ld_vol(c) < need) {
        if (++it > 8) __nanosleep(32);
        if ((it & 63u) == 1) {
            if (ddf_ld_relaxed_s32((const int32_t*)abort_flag) != 0) return false;
            if ((int64_t)(ddf_globaltimer() - t0) > cap_ns) {
                ddf_set_status(status, DDF_ERR_TIMEOUT);
                atomicExch(abort_flag, 1u);
                return false;
            }
        }
    }
    return true;
}

// 16-byte-granular range [a, z) of an array: aligned start, byte count, and
// the element shift of a inside the copied range.
struct Range16 {
    const unsigned char* src;
    uint32_t bytes;
    int32_t shift;
};
template <typename T>
__device__ __forceinline__ Range16 range16(const T* a, const T* z) {
    const uintptr_t pa = (uintptr_t)a, pz = (uintptr_t)z;
    const uintptr_t a16 = pa & ~(uintptr_t)15, z16 = (pz + 15) & ~(uintptr_t)15;
    return Range16{(const unsigned char*)a16, (uint32_t)(z16 - a16), (int32_t)((pa - a16) / sizeof(T))};
}

template <typename TV, typename TX>
__global__ void __launch_bounds__(DDF_BLK_CHAIN_LANES + 32 * BLK_PROD_MAX, 1)
k_sptrsv_blk(const int32_t* __restrict__ chunk_q0, const int32_t* __restrict__ chunk_meta,
             const int32_t* __restrict__ blk_chunk, const int32_t* __restrict__ esplit, int32_t n, int32_t nblocks,
             int32_t R, const int32_t* __restrict__ seq, const int32_t* __restrict__ st, const int32_t* __restrict__ col,
             const TV* __restrict__ val, const TX* __restrict__ dinv, const TX* __restrict__ b, TX* x,
             uint32_t* ticket, int32_t* status, int64_t cap_ns) {
    using B = XBits<TX>;
    using SL = SlotLayout<TV, TX>;
    extern __shared__ __align__(16) unsigned char blk_dsm[];
    TX* xs = reinterpret_cast<TX*>(blk_dsm);
    unsigned char* slots = blk_dsm + round16(R * (int)sizeof(TX));
    __shared__ BlkShared S;
    uint32_t* abort_flag = ticket + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nprod = (int)(blockDim.x >> 5) - BLK_CHAIN;
    if (threadIdx.x < nprod) mbar_init(&S.bar[threadIdx.x]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    uint32_t phase = 0;   // parity of this producer's slot barrier (kept across blocks)
    while (true) {
        if (threadIdx.x == 0) {
            S.blk = (int32_t)atomicAdd(ticket, 1u);
            S.chain_done = 0;
        }
        if (threadIdx.x < nprod) S.ext_done[threadIdx.x] = 0;
        __syncthreads();
        const int32_t blk = S.blk;
        if (blk >= nblocks) break;
        const int32_t base = blk * R;
        const int32_t c0 = blk_chunk[blk], nck = blk_chunk[blk + 1] - c0;
        if (warp >= BLK_CHAIN) {
            // ------------------------------ producer ------------------------------
            const int e = warp - BLK_CHAIN;
            unsigned char* slot = slots + (size_t)e * SL::BYTES;
            TV* svals = reinterpret_cast<TV*>(slot);
            int32_t* scols = reinterpret_cast<int32_t*>(slot + SL::VAL);
            int4* smeta = reinterpret_cast<int4*>(slot + SL::VAL + SL::COL);
            TX* sdinv = reinterpret_cast<TX*>(slot + SL::VAL + SL::COL + SL::META);
            // a wait that gave up ends this producer's work in the block: it
            // stages and publishes nothing more, so the chain's waits give up too
            for (int32_t k = e; k < nck; k += nprod) {
                if (k >= nprod) {
                    int ok = 1;
                    if (lane == 0) ok = wait_count(&S.chain_done, k - nprod + 1, status, abort_flag, cap_ns);
                    if (!__shfl_sync(0xffffffffu, ok, 0)) break;
                }
                const int32_t qa = chunk_q0[c0 + k], qb = chunk_q0[c0 + k + 1];
                const int32_t meta = chunk_meta[c0 + k];
                const bool direct = (meta & DDF_CK_DIRECT) != 0;
                const int32_t e0 = st[qa], e1 = st[qb];
                // stage the chunk's values and columns (one contiguous range each)
                Range16 rv{nullptr, 0, 0}, rc{nullptr, 0, 0};
                if (!direct && e1 > e0) {
                    rv = range16(val + e0, val + e1);
                    rc = range16(col + e0, col + e1);
                }
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(&S.bar[e], rv.bytes + rc.bytes);
                    if (rv.bytes) bulk_g2s(svals, rv.src, rv.bytes, &S.bar[e]);
                    if (rc.bytes) bulk_g2s(scols, rc.src, rc.bytes, &S.bar[e]);
                }
                // one lane per row while the copies fly: row (the plan's row map),
                // value extent, external count, 1 / L_ii; xs[r - base] = b[r]
                const int32_t rows = qb - qa;
                for (int32_t i = lane; i < rows; i += 32) {
                    const int32_t q = qa + i;
                    const int32_t r = seq[q], kb = st[q], L = st[q + 1] - kb, ns = esplit[q];
                    smeta[i] = make_int4(r - base, kb - e0, L, ns);
                    sdinv[i] = dinv[q];
                    xs[r - base] = b[r];
                }
                const bool landed = mbar_wait(&S.bar[e], phase, status, abort_flag, cap_ns);
                phase ^= 1u;
                if (!__all_sync(0xffffffffu, landed)) break;
                // v lanes per row: external sums; in-block columns become xs offsets
                const int v = DDF_CK_VPROD(meta);
                const int lg = __ffs(v) - 1, rpw = 32 >> lg, sub = lane >> lg, li = lane & (v - 1);
                for (int32_t ib = 0; ib < rows; ib += rpw) {
                    const int32_t i = ib + sub;
                    const bool act = i < rows;
                    TX acc = 0;
                    int32_t roff = 0;
                    if (act) {
                        const int4 m = smeta[i];
                        roff = m.x;
                        const int32_t kbl = m.y, L = m.z, ns = m.w;
                        for (int32_t i1b = 0; i1b < ns; i1b += BLK_PB * v) {
                            typename B::U xv[BLK_PB];
                            TX vv[BLK_PB];
                            int32_t jj[BLK_PB];
#pragma unroll
                            for (int t = 0; t < BLK_PB; ++t) {
                                const int32_t i1 = i1b + li + t * v;
                                jj[t] = -1;
                                vv[t] = 0;
                                if (i1 < ns) {
                                    jj[t] = direct ? col[e0 + kbl + i1] : scols[rc.shift + kbl + i1];
                                    vv[t] = ddf_cvt<TX>(direct ? val[e0 + kbl + i1] : svals[rv.shift + kbl + i1]);
                                    if ((uint32_t)jj[t] >= (uint32_t)n) {   // not a column: no read
                                        jj[t] = -1;
                                        acc = B::val(B::CANON);
                                    }
                                }
                            }
#pragma unroll
                            for (int t = 0; t < BLK_PB; ++t)
                                xv[t] = jj[t] >= 0 ? B::ld(x + jj[t]) : (typename B::U)0;
#pragma unroll
                            for (int t = 0; t < BLK_PB; ++t) {
                                if (jj[t] < 0) continue;
                                if (xv[t] == B::SENT) {
                                    TX w = wait_x<TX>(x + jj[t], status, abort_flag, cap_ns);
                                    xv[t] = B::bits(w) == B::SENT ? B::CANON : B::bits(w);
                                }
                                acc += vv[t] * B::val(xv[t]);
                            }
                        }
                        if (!direct)
                            for (int32_t i1 = ns + li; i1 < L; i1 += v) scols[rc.shift + kbl + i1] -= base;
                    }
                    for (int o = v >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (act && li == 0) xs[roff] -= acc;
                }
                if (lane == 0) {
                    S.crows[e] = rows;
                    S.cmeta[e] = meta;
                    S.dv[e] = rv.shift;
                    S.dc[e] = rc.shift;
                    S.e0[e] = e0;
                }
                __syncwarp();
                __threadfence_block();
                if (lane == 0) st_vol(&S.ext_done[e], k / nprod + 1);
            }
        } else {
            // ------------------------------- chain --------------------------------
            const int ct = threadIdx.x;   // 0 .. DDF_BLK_CHAIN_LANES - 1
            for (int32_t k = 0; k < nck; ++k) {
                const int e = k % nprod;
                int ok = 1;
                if (lane == 0) ok = wait_count(&S.ext_done[e], k / nprod + 1, status, abort_flag, cap_ns);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                __threadfence_block();
                const unsigned char* slot = slots + (size_t)e * SL::BYTES;
                const TV* svals = reinterpret_cast<const TV*>(slot);
                const int32_t* scols = reinterpret_cast<const int32_t*>(slot + SL::VAL);
                const int4* smeta = reinterpret_cast<const int4*>(slot + SL::VAL + SL::COL);
                const TX* sdinv = reinterpret_cast<const TX*>(slot + SL::VAL + SL::COL + SL::META);
                // the slot is read only after its producer published it; a warp whose
                // wait gave up takes the chunk's shape from the plan and skips the work
                const int32_t meta = ok ? S.cmeta[e] : chunk_meta[c0 + k];
                const int32_t rows = ok ? S.crows[e] : 0, dv = S.dv[e], dc = S.dc[e];
                if (!(meta & DDF_CK_DIRECT)) {
                    const int v = DDF_CK_VCHAIN(meta);
                    const int lg = __ffs(v) - 1, li = ct & (v - 1);
                    const int32_t slot_i = ct >> lg, stride = DDF_BLK_CHAIN_LANES >> lg, wslot = (warp * 32) >> lg;
                    for (int32_t ib = 0; ib + wslot < rows; ib += stride) {
                        const int32_t i = ib + slot_i;
                        const bool act = i < rows;
                        TX acc = 0, acc2 = 0;
                        int32_t roff = 0;
                        if (act) {
                            const int4 m = smeta[i];
                            roff = m.x;
                            const TV* pv = svals + dv + m.y;
                            const int32_t* pc = scols + dc + m.y;
                            // offsets of a valid plan lie in [0, R); anything else is
                            // read through the flag protocol (bounded).  Two sums in
                            // flight halve the dependent FMA chain.
                            auto xat = [&](int32_t o) -> TX {
                                if ((uint32_t)o < (uint32_t)R) return xs[o];
                                if ((uint32_t)(base + o) < (uint32_t)n) return dep<TX>(x, base + o, status, abort_flag, cap_ns);
                                return B::val(B::CANON);
                            };
                            int32_t i1 = m.w + li;
                            for (; i1 + v < m.z; i1 += 2 * v) {
                                acc += ddf_cvt<TX>(pv[i1]) * xat(pc[i1]);
                                acc2 += ddf_cvt<TX>(pv[i1 + v]) * xat(pc[i1 + v]);
                            }
                            if (i1 < m.z) acc += ddf_cvt<TX>(pv[i1]) * xat(pc[i1]);
                            acc += acc2;
                        }
                        for (int o = v >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                        if (act && li == 0) {
                            TX xr = (xs[roff] - acc) * sdinv[i];
                            typename B::U bits = B::bits(xr);
                            if (bits == B::SENT) bits = B::CANON;
                            xs[roff] = B::val(bits);
                            B::st(x + base + roff, bits);
                        }
                    }
                } else {
                    // one row longer than a slot: in-block points from global memory
                    const int4 m = ok ? smeta[0] : make_int4(0, 0, 0, 0);
                    const int32_t kb = S.e0[e] + m.y;
                    TX acc = 0;
                    for (int32_t i1 = m.w + ct; i1 < m.z; i1 += DDF_BLK_CHAIN_LANES) {
                        const int32_t j = col[kb + i1];
                        const TX xj = (uint32_t)(j - base) < (uint32_t)R ? xs[j - base]
                                      : (uint32_t)j < (uint32_t)n   ? dep<TX>(x, j, status, abort_flag, cap_ns)
                                                                    : B::val(B::CANON);
                        acc += ddf_cvt<TX>(val[kb + i1]) * xj;
                    }
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) S.red[warp] = (double)acc;
                    asm volatile("bar.sync 1, %0;" ::"n"(DDF_BLK_CHAIN_LANES) : "memory");
                    if (ct == 0 && ok) {
                        TX tot = 0;
                        for (int w = 0; w < BLK_CHAIN; ++w) tot += (TX)S.red[w];
                        TX xr = (xs[m.x] - tot) * sdinv[0];
                        typename B::U bits = B::bits(xr);
                        if (bits == B::SENT) bits = B::CANON;
                        xs[m.x] = B::val(bits);
                        B::st(x + base + m.x, bits);
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"n"(DDF_BLK_CHAIN_LANES) : "memory");
                if (ct == 0) st_vol(&S.chain_done, k + 1);
            }
        }
        __syncthreads();
    }
}

// Shared memory of the coarsened solve for R rows per block and `nprod` slots.
template <typename TV, typename TX>
size_t blocked_smem(int32_t R, int nprod) {
    return (size_t)round16(R * (int)sizeof(TX)) + (size_t)nprod * SlotLayout<TV, TX>::BYTES;
}

template <typename TV, typename TX>
ddf_status launch_blocked(ddf_plan_s* p, const TV* val, const TX* dinv, const TX* b, TX* x, cudaStream_t s) {
    const int32_t R = p->opts.coarsen_rows;
    auto kern = k_sptrsv_blk<TV, TX>;
    int optin = 0;
    DDF_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    cudaFuncAttributes fa;
    DDF_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    // as many producer warps (staging slots) as the shared memory left after xs holds
    int nprod = BLK_PROD_MAX;
    while (nprod > 1 && blocked_smem<TV, TX>(R, nprod) > room) --nprod;
    const size_t smem = blocked_smem<TV, TX>(R, nprod);
    if (smem > room) return DDF_ERR_ARG;
    const int threads = DDF_BLK_CHAIN_LANES + 32 * nprod;
    DDF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return DDF_ERR_CUDA;
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    int64_t ctas = std::min<int64_t>((int64_t)p->nblocks, (int64_t)per_sm * sm);
    kern<<<(unsigned)ctas, threads, smem, s>>>(p->chunk_q0, p->chunk_meta, p->blk_chunk, p->esplit, p->n,
                                               p->nblocks, R,
                                               p->seq, p->starts, p->col, val, dinv, b, x, p->ticket, p->status,
                                               p->opts.spin_cap_ns);
    ddf_count_launch();
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
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
    if (p->nblocks > 0 && p->n > 0) {
        ddf_status st = launch_blocked<TV, TX>(p, val, dinv, b, x, s);
        if (st) return st;
        ++launches;
    } else if (nu > 0) {
        int per_sm = 0;
        DDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sptrsv<TV, TX>, DDF_CTA_THREADS, 0));
        if (per_sm < 1) per_sm = 1;
        // Two CTAs per SM (16 warps) already exceed the units of one level of
        // the benchmark matrices; the rest of the SM stays free for work on
        // other streams.
        if (per_sm > DDF_SOLVE_CTAS_PER_SM) per_sm = DDF_SOLVE_CTAS_PER_SM;
        int64_t ctas = (nu + DDF_WARPS_PER_CTA - 1) / DDF_WARPS_PER_CTA;
        if (ctas > (int64_t)per_sm * sm) ctas = (int64_t)per_sm * sm;
        const dcod* a_cod = p->cod;
        const dunit* a_units = p->units[0];
        const int32_t* a_uq = p->unit_q;
        const int32_t* a_seq = p->seq;
        const int32_t* a_st = p->starts;
        const int32_t* a_col = p->col;
        uint32_t* a_ticket = p->ticket;
        int32_t* a_status = p->status;
        int64_t a_cap = p->opts.spin_cap_ns;
        void* args[] = {(void*)&a_cod, (void*)&a_units, (void*)&a_uq, (void*)&nu, (void*)&a_seq, (void*)&a_st, (void*)&a_col,
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
