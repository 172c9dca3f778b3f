// Batched and multi-RHS execution.
//
// A batch of independent matrices is inspected as one block-diagonal matrix:
// its partitions and codelets are those of Alg. 1 on that matrix, so every
// level of a batched SpTRSV holds the rows of all matrices at that level.
//
// The multi-RHS executors give a row of the block X ([n][nrhs], row-major)
// to a group of LP lanes: each lane moves VEC consecutive right-hand sides
// (16 bytes when nrhs = VEC * LP and the blocks are 16-byte aligned, else
// one element, LP = 32, lane k owning right-hand side k).  A row of at most
// SHORT_ROW points runs on one lane group (G = 32 / LP rows per warp at a
// time); a longer row runs on the whole warp, the G groups taking different
// points (one load instruction fetches the X rows of G points) and a
// butterfly over the groups combining their partial sums.  Every order is
// fixed, so results do not depend on timing.  The solve is a persistent grid
// of warps taking work items from a ticket; for a batch, its items are the
// plan's units split per matrix and long rows split into segments, handed out
// by normalized level (ddf_build_mrhs_items).  ddf_batch_run runs a batch's SpMV
// and SpTRSV in one launch.
#include <initializer_list>
#include <vector>

#include "ddf_internal.cuh"

namespace {

constexpr int NRHS_MAX = 32;

__global__ void k_add_offset(int32_t* __restrict__ a, int64_t n, int32_t add) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += add;
}

// Bits of one element of X: the fill pattern that marks "not solved yet" and
// the canonical NaN a solved element takes if its bits equal the pattern.
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
    static __device__ __forceinline__ U bits(float v) { return (U)__float_as_uint(v); }
};

// Access to VEC consecutive right-hand sides of one row of X: plain reads
// (SpMM), relaxed reads and writes of the ready-flag protocol (SpTRSM).
template <typename TX, int VEC>
struct VA;
template <typename TX>
struct VA<TX, 1> {
    using U = typename RB<TX>::U;
    static __device__ __forceinline__ void ld_nc(const TX* p, TX (&o)[1]) { o[0] = __ldg(p); }
    static __device__ __forceinline__ void st(TX* p, const TX (&v)[1]) { *p = v[0]; }
    static __device__ __forceinline__ void ld_relaxed(const void* p, U (&o)[1]) { o[0] = RB<TX>::ld(p); }
    static __device__ __forceinline__ void st_relaxed(void* p, const U (&v)[1]) { RB<TX>::st(p, v[0]); }
};
template <>
struct VA<float, 4> {
    using U = uint32_t;
    static __device__ __forceinline__ void ld_nc(const float* p, float (&o)[4]) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = t.x;
        o[1] = t.y;
        o[2] = t.z;
        o[3] = t.w;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    static __device__ __forceinline__ void ld_relaxed(const void* p, U (&o)[4]) {
        asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3])
                     : "l"(p)
                     : "memory");
    }
    static __device__ __forceinline__ void st_relaxed(void* p, const U (&v)[4]) {
        asm volatile("st.relaxed.gpu.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v[0]), "r"(v[1]),
                     "r"(v[2]), "r"(v[3])
                     : "memory");
    }
};
template <>
struct VA<double, 2> {
    using U = unsigned long long;
    static __device__ __forceinline__ void ld_nc(const double* p, double (&o)[2]) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = t.x;
        o[1] = t.y;
    }
    static __device__ __forceinline__ void st(double* p, const double (&v)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
    static __device__ __forceinline__ void ld_relaxed(const void* p, U (&o)[2]) {
        asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(o[0]), "=l"(o[1]) : "l"(p) : "memory");
    }
    static __device__ __forceinline__ void st_relaxed(void* p, const U (&v)[2]) {
        asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(v[0]), "l"(v[1]) : "memory");
    }
};

// Lane layout of the executors: VEC elements per lane, LP lanes per row of
// X, G groups per warp, NL loads per lane in flight together, SUB points
// covered by them.
template <typename TX, int VEC_, int LP_>
struct Lay {
    static constexpr int VEC = VEC_, LP = LP_, G = 32 / LP_, NL = LP_ < 8 ? LP_ : 8, SUB = NL * (32 / LP_);
    using V = VA<TX, VEC_>;
};

// sum over the G lane groups; afterwards every group holds the row's total
template <typename TX, int LP, int VEC>
__device__ __forceinline__ void group_sum(TX (&acc)[VEC]) {
#pragma unroll
    for (int off = LP; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
}

// Column of point i1 of row i0 of codelet C (the three access functions of h).
__device__ __forceinline__ int32_t point_col(const dcod& C, const int32_t* __restrict__ col, int32_t i0,
                                             int32_t kb, int32_t i1) {
    const int32_t hb = C.h0 + C.delta * i0;
    if (C.type == DDF_BLAS) return hb + C.sigma * i1;
    if (C.type == DDF_PSC1) return hb + (col[C.sref + i1] - C.h0);
    return col[kb + i1];
}

// ---------------------------------------------------------------------------
// SpMM: Y = A X over the SpMV plan's work units and value tiles
// ---------------------------------------------------------------------------

// A row of the multi-RHS SpMV: its first 32 points (lane t: point t's value
// and column), its value extent, and the row of Y it writes.  Point i1's value
// is val[kb + i1 * vs] (vs > 1 for rows of SpMV value tiles).
template <typename TX>
struct SRow {
    int32_t kb, L, vs, pj, f;
    TX pv;
};

template <typename TV, typename TX>
__device__ __forceinline__ void srow_point(const dcod& C, int32_t i0, int32_t kb, int32_t L, int32_t vs,
                                           int32_t i1, const int32_t* __restrict__ col,
                                           const TV* __restrict__ val, TX& pv, int32_t& pj) {
    pv = (TX)0;
    pj = 0;
    if (i1 < L) {
        pv = ddf_cvt<TX>(__ldcs(val + kb + (int64_t)i1 * vs));
        pj = point_col(C, col, i0, kb, i1);
    }
}

template <typename TV, typename TX>
__device__ __forceinline__ void srow_load(const dcod& C, int32_t i0, bool act, const int32_t* __restrict__ st,
                                          const int32_t* __restrict__ col, const TV* __restrict__ val, int lane,
                                          int32_t vs, int32_t vb, SRow<TX>& m) {
    m.kb = m.L = m.pj = m.f = 0;
    m.vs = vs;
    m.pv = (TX)0;
    if (!act) return;
    const int32_t q = C.q0 + i0;
    if (C.type == DDF_PSC2) {
        m.kb = st[q];
        m.L = st[q + 1] - m.kb;
    } else {
        m.kb = vb >= 0 ? vb : C.g0 + C.gamma * i0;
        m.L = C.n;
    }
    m.f = C.f0 + C.rho * i0;
    srow_point<TV, TX>(C, i0, m.kb, m.L, vs, lane, col, val, m.pv, m.pj);
}

// y_r = sum over the row's points of a * x_col
template <typename TV, typename TX, class LY>
__device__ __forceinline__ void srow_compute(const dcod& C, int32_t i0, const SRow<TX>& m,
                                             const int32_t* __restrict__ col, const TV* __restrict__ val,
                                             const TX* __restrict__ X, TX* __restrict__ Y, int32_t nrhs, int lane) {
    using V = typename LY::V;
    constexpr int VEC = LY::VEC, G = LY::G, NL = LY::NL, SUB = LY::SUB;
    const int g = lane / LY::LP, c = lane % LY::LP;
    const bool on = c * VEC < nrhs;
    TX acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = (TX)0;
    TX pv = m.pv;
    int32_t pj = m.pj;
    for (int32_t p0 = 0; p0 < m.L; p0 += 32) {
        TX npv = (TX)0;
        int32_t npj = 0;
        if (p0 + 32 < m.L) srow_point<TV, TX>(C, i0, m.kb, m.L, m.vs, p0 + 32 + lane, col, val, npv, npj);
        const int32_t cnt = min(32, m.L - p0);
        for (int32_t s0 = 0; s0 < cnt; s0 += SUB) {
            TX xv[NL][VEC];
            TX av[NL];
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                const int t = s0 + k * G + g;
                av[k] = __shfl_sync(0xffffffffu, pv, t & 31);
                const int32_t j = __shfl_sync(0xffffffffu, pj, t & 31);
                if (on && t < cnt) {
                    V::ld_nc(X + (int64_t)j * nrhs + c * VEC, xv[k]);
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) xv[k][v] = (TX)0;
                }
            }
#pragma unroll
            for (int k = 0; k < NL; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] += av[k] * xv[k][v];
        }
        pv = npv;
        pj = npj;
    }
    group_sum<TX, LY::LP, VEC>(acc);
    if (g == 0 && on) V::st(Y + (int64_t)m.f * nrhs + c * VEC, acc);
}

// A row of at most SHORT_ROW points on one lane group (group g of LP lanes):
// the group walks the row's points NB at a time, lane c < NB loading point
// p0 + c's value and column, every lane reading its VEC right-hand sides of
// each point's X row; the group writes its row of Y.  The group's shuffles
// name only its own lanes.
constexpr int SHORT_ROW = 32;

template <typename TV, typename TX, class LY>
__device__ __forceinline__ void gspmm_row(const dcod& C, int32_t i0, int32_t kb, int32_t L, int32_t vs, int32_t f,
                                          const int32_t* __restrict__ col, const TV* __restrict__ val,
                                          const TX* __restrict__ X, TX* __restrict__ Y, int32_t nrhs, int g,
                                          int c) {
    using V = typename LY::V;
    constexpr int VEC = LY::VEC, LP = LY::LP, NB = LY::NL;
    const unsigned gmask = ((1u << LP) - 1u) << (g * LP);
    TX acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = (TX)0;
    for (int32_t p0 = 0; p0 < L; p0 += NB) {
        TX pv = (TX)0;
        int32_t pj = 0;
        if (c < NB && p0 + c < L) {
            pv = ddf_cvt<TX>(__ldcs(val + kb + (int64_t)(p0 + c) * vs));
            pj = point_col(C, col, i0, kb, p0 + c);
        }
        const int32_t cnt = min(NB, L - p0);
        TX xv[NB][VEC];
        TX av[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            av[t] = __shfl_sync(gmask, pv, t, LP);
            const int32_t j = __shfl_sync(gmask, pj, t, LP);
            if (t < cnt) {
                V::ld_nc(X + (int64_t)j * nrhs + c * VEC, xv[t]);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) xv[t][v] = (TX)0;
            }
        }
#pragma unroll
        for (int t = 0; t < NB; ++t)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += av[t] * xv[t][v];
    }
    V::st(Y + (int64_t)f * nrhs + c * VEC, acc);
}

// Value extent of row i0 of codelet C (vb >= 0: a tile row, values at vb + i1 vs).
__device__ __forceinline__ void spmm_row_extent(const dcod& C, int32_t i0, int32_t vb,
                                                const int32_t* __restrict__ st, int32_t& kb, int32_t& L) {
    if (C.type == DDF_PSC2) {
        const int32_t q = C.q0 + i0;
        kb = st[q];
        L = st[q + 1] - kb;
    } else {
        kb = vb >= 0 ? vb : C.g0 + C.gamma * i0;
        L = C.n;
    }
}

// Operands of the multi-RHS SpMV: the plan's codelets, rows (starts, col),
// values, work units and value tiles, and the blocks X and Y.
template <typename TV, typename TX>
struct MulArgs {
    const dcod* cod;
    const int32_t* st;
    const int32_t* col;
    const TV* val;
    const TX* X;
    TX* Y;
    int32_t nrhs;
    const dunit* units[3];
    int64_t nunits[3];
    const dtile* tiles[2];
    int64_t ntiles[2];
};

// One work unit on one warp.  Element-per-lane layout: rows in pairs, the
// next row's points loading while the current row's X rows are read.
// 16-byte layout: G rows at a time, one per lane group when all have at most
// SHORT_ROW points, else one after another on the whole warp.
template <typename TV, typename TX, class LY>
__device__ __forceinline__ void spmm_unit(const MulArgs<TV, TX>& A, const dunit& U, int lane) {
    constexpr int G = LY::G, LP = LY::LP;
    const int g = lane / LP, c = lane % LP;
    const int32_t ncods = U.i0b < 0 ? -U.i0b : 1;
    for (int32_t k = 0; k < ncods; ++k) {
        const dcod C = A.cod[U.cod + k];
        const int32_t b0 = U.i0b < 0 ? 0 : U.i0b;
        const int32_t e0 = U.i0b < 0 ? C.m : U.i0e;
        if constexpr (LP == 32) {
            SRow<TX> ma, mb;
            srow_load<TV, TX>(C, b0, b0 < e0, A.st, A.col, A.val, lane, 1, -1, ma);
            for (int32_t i0 = b0; i0 < e0; i0 += 2) {
                srow_load<TV, TX>(C, i0 + 1, i0 + 1 < e0, A.st, A.col, A.val, lane, 1, -1, mb);
                srow_compute<TV, TX, LY>(C, i0, ma, A.col, A.val, A.X, A.Y, A.nrhs, lane);
                if (i0 + 1 >= e0) break;
                srow_load<TV, TX>(C, i0 + 2, i0 + 2 < e0, A.st, A.col, A.val, lane, 1, -1, ma);
                srow_compute<TV, TX, LY>(C, i0 + 1, mb, A.col, A.val, A.X, A.Y, A.nrhs, lane);
            }
        } else {
            for (int32_t i0 = b0; i0 < e0; i0 += G) {
                const int32_t i = i0 + g;
                int32_t kb = 0, L = 0;
                if (i < e0) spmm_row_extent(C, i, -1, A.st, kb, L);
                if (!__any_sync(0xffffffffu, L > SHORT_ROW)) {
                    if (i < e0)
                        gspmm_row<TV, TX, LY>(C, i, kb, L, 1, C.f0 + C.rho * i, A.col, A.val, A.X, A.Y, A.nrhs, g,
                                              c);
                } else {
                    for (int32_t h = i0; h < min(i0 + G, e0); ++h) {
                        SRow<TX> m;
                        srow_load<TV, TX>(C, h, true, A.st, A.col, A.val, lane, 1, -1, m);
                        srow_compute<TV, TX, LY>(C, h, m, A.col, A.val, A.X, A.Y, A.nrhs, lane);
                    }
                }
            }
        }
    }
}

// One value tile (point-major values of up to 8 rows) on one warp, rows laid
// out over the lanes as in spmm_unit.
template <typename TV, typename TX, class LY>
__device__ __forceinline__ void spmm_tile(const MulArgs<TV, TX>& A, const dtile& T, int lane) {
    constexpr int G = LY::G, LP = LY::LP;
    const int g = lane / LP, c = lane % LP;
    const int32_t w = (int32_t)(T.meta & 7u) + 1;
    auto codelet = [&](int32_t r) { return A.cod[T.cod + (int32_t)((T.meta >> (3 + 3 * r)) & 7u)]; };
    if constexpr (LP == 32) {
        SRow<TX> ma, mb;
        dcod Ca = codelet(0), Cb = Ca;
        srow_load<TV, TX>(Ca, T.q - Ca.q0, true, A.st, A.col, A.val, lane, w, T.vb, ma);
        for (int32_t r = 0; r < w; r += 2) {
            if (r + 1 < w) {
                Cb = codelet(r + 1);
                srow_load<TV, TX>(Cb, T.q + r + 1 - Cb.q0, true, A.st, A.col, A.val, lane, w, T.vb + r + 1, mb);
            }
            srow_compute<TV, TX, LY>(Ca, T.q + r - Ca.q0, ma, A.col, A.val, A.X, A.Y, A.nrhs, lane);
            if (r + 1 >= w) break;
            if (r + 2 < w) {
                Ca = codelet(r + 2);
                srow_load<TV, TX>(Ca, T.q + r + 2 - Ca.q0, true, A.st, A.col, A.val, lane, w, T.vb + r + 2, ma);
            }
            srow_compute<TV, TX, LY>(Cb, T.q + r + 1 - Cb.q0, mb, A.col, A.val, A.X, A.Y, A.nrhs, lane);
        }
    } else {
        for (int32_t r0 = 0; r0 < w; r0 += G) {
            const int32_t r = r0 + g;
            const dcod C = codelet(min(r, w - 1));
            const int32_t i = T.q + r - C.q0;
            const int32_t L = r < w ? C.n : 0;   // tile rows are BLAS / PSC I rows of C.n points
            if (!__any_sync(0xffffffffu, L > SHORT_ROW)) {
                if (r < w)
                    gspmm_row<TV, TX, LY>(C, i, T.vb + r, L, w, C.f0 + C.rho * i, A.col, A.val, A.X, A.Y, A.nrhs, g,
                                          c);
            } else {
                for (int32_t h = r0; h < min(r0 + G, w); ++h) {
                    const dcod Ch = codelet(h);
                    SRow<TX> m;
                    srow_load<TV, TX>(Ch, T.q + h - Ch.q0, true, A.st, A.col, A.val, lane, w, T.vb + h, m);
                    srow_compute<TV, TX, LY>(Ch, T.q + h - Ch.q0, m, A.col, A.val, A.X, A.Y, A.nrhs, lane);
                }
            }
        }
    }
}

// Work unit array k (k < 3) or tile array k - 3 of the plan, one warp per item.
// The products are bound by L2 latency: four resident CTAs per SM (64
// registers a thread, a few spilled) measured faster than three.
constexpr int SPMM_MIN_CTAS = 4;

template <typename TV, typename TX, class LY>
__global__ void __launch_bounds__(DDF_CTA_THREADS, SPMM_MIN_CTAS) k_spmm(MulArgs<TV, TX> A, int k) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = k < 3 ? A.nunits[k] : A.ntiles[k - 3];
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < count; u += nw) {
        if (k < 3) spmm_unit<TV, TX, LY>(A, A.units[k][u], lane);
        else spmm_tile<TV, TX, LY>(A, A.tiles[k - 3][u], lane);
    }
}

// ---------------------------------------------------------------------------
// SpTRSM: L X = B over the SpTRSV plan, one row per warp at a time
// ---------------------------------------------------------------------------

template <typename U>
__global__ void k_fill_m(U* __restrict__ x, int64_t n, U pattern, uint32_t* __restrict__ ticket) {
    int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        ticket[0] = 0u;
        ticket[1] = 0u;
    }
    for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = pattern;
}

// Waits until none of the loaded X entries xb[t] (points t < cnt) holds the
// fill pattern: the X rows of every point still pending are read again, all
// together, each round, so a row waits for its latest dependency plus one
// round trip rather than for each pending point in turn.  Bounded: after
// cap_ns (or once another warp gave up) the pending entries become NaN and
// the status word records DDF_ERR_TIMEOUT.
template <class V, typename TX, int NB, int VEC>
__device__ __forceinline__ void settle(typename V::U (&xb)[NB][VEC], const int32_t (&jv)[NB], int32_t cnt,
                                       const TX* X, int32_t nrhs, int c, int32_t* status, uint32_t* abort_flag,
                                       int64_t cap_ns) {
    using RBx = RB<TX>;
    uint32_t pend = 0;
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
        for (int v = 0; v < VEC; ++v)
            if (t < cnt && xb[t][v] == RBx::SENT) pend |= 1u << t;
    if (!pend) return;
    const uint64_t t0 = ddf_globaltimer();
    for (uint32_t it = 1;; ++it) {
#pragma unroll
        for (int t = 0; t < NB; ++t)
            if ((pend >> t) & 1u) V::ld_relaxed(X + (int64_t)jv[t] * nrhs + c * VEC, xb[t]);
        uint32_t still = 0;
#pragma unroll
        for (int t = 0; t < NB; ++t)
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                if (((pend >> t) & 1u) && xb[t][v] == RBx::SENT) still |= 1u << t;
        pend = still;
        if (!pend) return;
        if ((it & 15u) == 0) {
            bool give_up = ddf_ld_relaxed_s32(abort_flag) != 0;
            if (!give_up && (int64_t)(ddf_globaltimer() - t0) > cap_ns) {
                ddf_set_status(status, DDF_ERR_TIMEOUT);
                atomicExch(abort_flag, 1u);
                give_up = true;
            }
            if (give_up) {
#pragma unroll
                for (int t = 0; t < NB; ++t)
#pragma unroll
                    for (int v = 0; v < VEC; ++v)
                        if (((pend >> t) & 1u) && xb[t][v] == RBx::SENT) xb[t][v] = RBx::CANON;
                return;
            }
        }
        if (it > 8) __nanosleep(64);
    }
}

// What a row of the solve needs before its dependencies: its row r, value
// extent, the lane's entries of b, 1 / L_rr, and lane t's point t (value and
// column) of its first 32 points.  The plan keeps every position's
// off-diagonal points in level order (starts, col, val), whatever the type of
// the codelet holding it, so the solve reads rows without the codelets.
template <typename TX, int VEC>
struct QRow {
    int32_t r, kb, L, pj;
    TX di, pv;
    TX bv[VEC];
};

template <typename TV, typename TX, class LY>
__device__ __forceinline__ void qrow_load(int64_t q, bool act, const int32_t* __restrict__ seq,
                                          const int32_t* __restrict__ st, const int32_t* __restrict__ col,
                                          const TV* __restrict__ val, const TX* __restrict__ dinv,
                                          const TX* __restrict__ B, int32_t nrhs, int lane,
                                          QRow<TX, LY::VEC>& m) {
    constexpr int VEC = LY::VEC;
    m.r = m.kb = m.L = m.pj = 0;
    m.di = m.pv = (TX)0;
#pragma unroll
    for (int v = 0; v < VEC; ++v) m.bv[v] = (TX)0;
    if (!act) return;
    m.r = seq[q];
    m.kb = st[q];
    m.L = st[q + 1] - m.kb;
    m.di = dinv[q];
    const int c = lane % LY::LP;
    if (c * VEC < nrhs) LY::V::ld_nc(B + (int64_t)m.r * nrhs + c * VEC, m.bv);
    if (lane < m.L) {
        m.pv = ddf_cvt<TX>(val[m.kb + lane]);
        m.pj = col[m.kb + lane];
    }
}

// One row: the loads of a sub-block of points (NL per lane, G points per
// load) are all issued before any is checked, so one L2 round trip covers
// SUB points of the row; an element still holding the fill pattern is
// waited on (bounded) before it is used.
template <typename TV, typename TX, class LY>
__device__ __forceinline__ void qrow_solve(const QRow<TX, LY::VEC>& m, const int32_t* __restrict__ col,
                                           const TV* __restrict__ val, TX* X, int32_t nrhs, int lane,
                                           int32_t* status, uint32_t* abort_flag, int64_t cap_ns) {
    using V = typename LY::V;
    using RBx = RB<TX>;
    using U = typename V::U;
    constexpr int VEC = LY::VEC, G = LY::G, NL = LY::NL, SUB = LY::SUB;
    const int g = lane / LY::LP, c = lane % LY::LP;
    const bool on = c * VEC < nrhs;
    TX acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = (TX)0;
    TX pv = m.pv;
    int32_t pj = m.pj;
    for (int32_t p0 = 0; p0 < m.L; p0 += 32) {
        TX npv = (TX)0;
        int32_t npj = 0;
        if (p0 + 32 + lane < m.L) {
            npv = ddf_cvt<TX>(val[m.kb + p0 + 32 + lane]);
            npj = col[m.kb + p0 + 32 + lane];
        }
        const int32_t cnt = min(32, m.L - p0);
        for (int32_t s0 = 0; s0 < cnt; s0 += SUB) {
            U xb[NL][VEC];
            TX av[NL];
            int32_t jv[NL];
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                const int t = s0 + k * G + g;
                av[k] = __shfl_sync(0xffffffffu, pv, t & 31);
                jv[k] = __shfl_sync(0xffffffffu, pj, t & 31);
                if (on && t < cnt) {
                    V::ld_relaxed(X + (int64_t)jv[k] * nrhs + c * VEC, xb[k]);
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) xb[k][v] = (U)0;
                }
            }
            if (on) {
                // the sub-block's points held by this lane: t = s0 + k G + g < cnt
                const int32_t mine = cnt > s0 + g ? (cnt - s0 - g + G - 1) / G : 0;
                settle<V, TX, NL, VEC>(xb, jv, mine, X, nrhs, c, status, abort_flag, cap_ns);
#pragma unroll
                for (int k = 0; k < NL; ++k)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] += av[k] * RBx::val(xb[k][v]);
            }
        }
        pv = npv;
        pj = npj;
    }
    group_sum<TX, LY::LP, VEC>(acc);
    if (g == 0 && on) {
        U bits[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            bits[v] = RBx::bits((m.bv[v] - acc[v]) * m.di);
            if (bits[v] == RBx::SENT) bits[v] = RBx::CANON;
        }
        V::st_relaxed(X + (int64_t)m.r * nrhs + c * VEC, bits);
    }
}

// A short row (at most SHORT_ROW points) solved by its own lane group: the
// LP lanes of group g hold row q's data (QRow, lane c = lane % LP loading
// point c of each block of NB points), and the group walks the row's points
// NB at a time, every lane reading its VEC right-hand sides of each point's
// X row: NB loads per lane in flight together, no cross-lane reduction.  The
// group's shuffles name only its own lanes, so a group waiting on a
// dependency does not hold the others back.

template <typename TV, typename TX, class LY>
__device__ __forceinline__ void grow_load(int64_t q, bool act, const int32_t* __restrict__ seq,
                                          const int32_t* __restrict__ st, const int32_t* __restrict__ col,
                                          const TV* __restrict__ val, const TX* __restrict__ dinv,
                                          const TX* __restrict__ B, int32_t nrhs, int c, QRow<TX, LY::VEC>& m) {
    constexpr int VEC = LY::VEC, NB = LY::NL;
    m.r = m.kb = m.L = m.pj = 0;
    m.di = m.pv = (TX)0;
#pragma unroll
    for (int v = 0; v < VEC; ++v) m.bv[v] = (TX)0;
    if (!act) return;
    m.r = seq[q];
    m.kb = st[q];
    m.L = st[q + 1] - m.kb;
    m.di = dinv[q];
    LY::V::ld_nc(B + (int64_t)m.r * nrhs + c * VEC, m.bv);
    if (c < NB && c < m.L) {
        m.pv = ddf_cvt<TX>(val[m.kb + c]);
        m.pj = col[m.kb + c];
    }
}

template <typename TV, typename TX, class LY>
__device__ __forceinline__ void grow_solve(const QRow<TX, LY::VEC>& m, const int32_t* __restrict__ col,
                                           const TV* __restrict__ val, TX* X, int32_t nrhs, int g, int c,
                                           int32_t* status, uint32_t* abort_flag, int64_t cap_ns) {
    using V = typename LY::V;
    using RBx = RB<TX>;
    using U = typename V::U;
    constexpr int VEC = LY::VEC, LP = LY::LP, NB = LY::NL;
    const unsigned gmask = (LP == 32) ? 0xffffffffu : (((1u << LP) - 1u) << (g * LP));
    TX acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = (TX)0;
    TX pv = m.pv;
    int32_t pj = m.pj;
    for (int32_t p0 = 0; p0 < m.L; p0 += NB) {
        if (p0 > 0) {
            pv = (TX)0;
            pj = 0;
            if (c < NB && p0 + c < m.L) {
                pv = ddf_cvt<TX>(val[m.kb + p0 + c]);
                pj = col[m.kb + p0 + c];
            }
        }
        const int32_t cnt = min(NB, m.L - p0);
        U xb[NB][VEC];
        TX av[NB];
        int32_t jv[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            av[t] = __shfl_sync(gmask, pv, t, LP);
            jv[t] = __shfl_sync(gmask, pj, t, LP);
            if (t < cnt) {
                V::ld_relaxed(X + (int64_t)jv[t] * nrhs + c * VEC, xb[t]);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) xb[t][v] = (U)0;
            }
        }
        settle<V, TX, NB, VEC>(xb, jv, cnt, X, nrhs, c, status, abort_flag, cap_ns);
#pragma unroll
        for (int t = 0; t < NB; ++t)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += av[t] * RBx::val(xb[t][v]);
    }
    U bits[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        bits[v] = RBx::bits((m.bv[v] - acc[v]) * m.di);
        if (bits[v] == RBx::SENT) bits[v] = RBx::CANON;
    }
    V::st_relaxed(X + (int64_t)m.r * nrhs + c * VEC, bits);
}

constexpr int SPTRSM_MIN_CTAS = 2;   // resident CTAs per SM the register budget is cut for
constexpr int SEG_POINTS = 64;       // batch solve: rows of more points run as segments on several warps

// Operands of the multi-RHS solve: its work ranges (the plan's units, or for
// a batch the units split where the matrix changes: first positions, and the
// ticket order), the plan's level-ordered rows (seq, starts, col, values,
// 1 / L_rr), the blocks B and X, the ticket (ticket[0]; ticket[1] is the
// give-up flag), the status word and the wait limit.
template <typename TV, typename TX>
struct SolveArgs {
    int32_t n;
    int64_t nunits;
    int32_t upt;
    const int32_t* order;   // items in ticket order (NULL: level order)
    const int32_t* unit_q;
    const int2* seg;        // per item: (segment, first partial-sum slot), x = -1 for a range; NULL: no segments
    TX* part;               // partial sums, NRHS_MAX per slot
    uint32_t* cnt;          // segments finished, per long row
    const int32_t* seq;
    const int32_t* st;
    const int32_t* col;
    const TV* val;
    const TX* dinv;
    const TX* B;
    TX* X;
    int32_t nrhs;
    uint32_t* ticket;
    int32_t* status;
    int64_t cap_ns;
};

// Segment s of the long row at position q (points s SEG_POINTS .. s
// SEG_POINTS + SEG_POINTS - 1) on one warp: its partial sums go to slot
// g0 + s; the warp that finishes the row's last segment adds the slots in
// segment order, solves the row and resets the row's counter for the next
// solve.  Segments never wait on one another, so the ticket argument holds.
template <typename TV, typename TX, class LY>
__device__ __forceinline__ void solve_segment(const SolveArgs<TV, TX>& A, int64_t q, int32_t s, int32_t g0,
                                              int lane) {
    using V = typename LY::V;
    using RBx = RB<TX>;
    using U = typename V::U;
    constexpr int VEC = LY::VEC, G = LY::G, NL = LY::NL, SUB = LY::SUB;
    const int g = lane / LY::LP, c = lane % LY::LP;
    const bool on = c * VEC < A.nrhs;
    uint32_t* abort_flag = A.ticket + 1;
    const int32_t kb = A.st[q], L = A.st[q + 1] - kb;
    const int32_t S = (L + SEG_POINTS - 1) / SEG_POINTS;
    const int32_t pb = s * SEG_POINTS, pe = min(L, pb + SEG_POINTS);
    TX acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = (TX)0;
    for (int32_t p0 = pb; p0 < pe; p0 += 32) {
        TX pv = (TX)0;
        int32_t pj = 0;
        if (p0 + lane < pe) {
            pv = ddf_cvt<TX>(A.val[kb + p0 + lane]);
            pj = A.col[kb + p0 + lane];
        }
        const int32_t cnt = min(32, pe - p0);
        for (int32_t s0 = 0; s0 < cnt; s0 += SUB) {
            U xb[NL][VEC];
            TX av[NL];
            int32_t jv[NL];
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                const int t = s0 + k * G + g;
                av[k] = __shfl_sync(0xffffffffu, pv, t & 31);
                jv[k] = __shfl_sync(0xffffffffu, pj, t & 31);
                if (on && t < cnt) {
                    V::ld_relaxed(A.X + (int64_t)jv[k] * A.nrhs + c * VEC, xb[k]);
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) xb[k][v] = (U)0;
                }
            }
            if (on) {
                const int32_t mine = cnt > s0 + g ? (cnt - s0 - g + G - 1) / G : 0;
                settle<V, TX, NL, VEC>(xb, jv, mine, A.X, A.nrhs, c, A.status, abort_flag, A.cap_ns);
#pragma unroll
                for (int k = 0; k < NL; ++k)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] += av[k] * RBx::val(xb[k][v]);
            }
        }
    }
    group_sum<TX, LY::LP, VEC>(acc);
    if (g == 0 && on) {
        U bits[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) bits[v] = RBx::bits(acc[v]);
        V::st_relaxed(A.part + (int64_t)(g0 + s) * NRHS_MAX + c * VEC, bits);
    }
    __syncwarp();
    __threadfence();
    uint32_t done = 0;
    if (lane == 0) done = atomicAdd(A.cnt + g0, 1u);
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done != (uint32_t)(S - 1)) return;
    __threadfence();
    if (g == 0 && on) {
        TX tot[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) tot[v] = (TX)0;
        for (int32_t k = 0; k < S; ++k) {
            U pb2[VEC];
            V::ld_relaxed(A.part + (int64_t)(g0 + k) * NRHS_MAX + c * VEC, pb2);
#pragma unroll
            for (int v = 0; v < VEC; ++v) tot[v] += RBx::val(pb2[v]);
        }
        const int32_t r = A.seq[q];
        const TX di = A.dinv[q];
        TX bv[VEC];
        V::ld_nc(A.B + (int64_t)r * A.nrhs + c * VEC, bv);
        U bits[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            bits[v] = RBx::bits((bv[v] - tot[v]) * di);
            if (bits[v] == RBx::SENT) bits[v] = RBx::CANON;
        }
        V::st_relaxed(A.X + (int64_t)r * A.nrhs + c * VEC, bits);
    }
    if (lane == 0) A.cnt[g0] = 0u;
}

// Ranges at ticket positions u0 .. u1 - 1 of the solve on one warp, in order.
// Inside a range (rows of one codelet, so of one level: they never read one
// another), G rows at a time: when all of them have at most SHORT_ROW
// points, one row per lane group; otherwise one row after another on the
// whole warp, the G groups splitting each row's points.  The next rows' data load while the current
// ones are solved.  Row x[r] is ready once its elements no longer hold the
// fill pattern; each lane waits on its own elements.
template <typename TV, typename TX, class LY>
__device__ __forceinline__ void solve_units(const SolveArgs<TV, TX>& A, int64_t u0, int64_t u1, int lane) {
    constexpr int G = LY::G, LP = LY::LP, VEC = LY::VEC;
    const int g = lane / LP, c = lane % LP;
    uint32_t* abort_flag = A.ticket + 1;
    for (int64_t i = u0; i < u1; ++i) {
        const int64_t u = A.order ? (int64_t)A.order[i] : i;
        if (A.seg) {
            const int2 sg = A.seg[u];
            if (sg.x >= 0) {
                solve_segment<TV, TX, LY>(A, A.unit_q[u], sg.x, sg.y, lane);
                continue;
            }
        }
        const int64_t qa = A.unit_q[u];
        const int64_t qz = (u + 1 < A.nunits) ? (int64_t)A.unit_q[u + 1] : (int64_t)A.n;
        if constexpr (LP == 32) {
            // one element per lane: rows one after another, points split over the warp
            QRow<TX, VEC> ma, mb;
            int64_t q = qa;
            qrow_load<TV, TX, LY>(q, q < qz, A.seq, A.st, A.col, A.val, A.dinv, A.B, A.nrhs, lane, ma);
            for (; q < qz; q += 2) {
                qrow_load<TV, TX, LY>(q + 1, q + 1 < qz, A.seq, A.st, A.col, A.val, A.dinv, A.B, A.nrhs, lane, mb);
                qrow_solve<TV, TX, LY>(ma, A.col, A.val, A.X, A.nrhs, lane, A.status, abort_flag, A.cap_ns);
                if (q + 1 >= qz) break;
                qrow_load<TV, TX, LY>(q + 2, q + 2 < qz, A.seq, A.st, A.col, A.val, A.dinv, A.B, A.nrhs, lane, ma);
                qrow_solve<TV, TX, LY>(mb, A.col, A.val, A.X, A.nrhs, lane, A.status, abort_flag, A.cap_ns);
            }
        } else {
            QRow<TX, VEC> cur, nxt;
            grow_load<TV, TX, LY>(qa + g, qa + g < qz, A.seq, A.st, A.col, A.val, A.dinv, A.B, A.nrhs, c, cur);
            for (int64_t s0 = qa; s0 < qz; s0 += G) {
                grow_load<TV, TX, LY>(s0 + G + g, s0 + G + g < qz, A.seq, A.st, A.col, A.val, A.dinv, A.B, A.nrhs,
                                      c, nxt);
                if (!__any_sync(0xffffffffu, cur.L > SHORT_ROW)) {
                    if (s0 + g < qz)
                        grow_solve<TV, TX, LY>(cur, A.col, A.val, A.X, A.nrhs, g, c, A.status, abort_flag, A.cap_ns);
                } else {
                    // the G rows in order on the whole warp; row h's data comes from group h
                    for (int h = 0; h < G; ++h) {
                        if (s0 + h >= qz) break;
                        QRow<TX, VEC> m;
                        const int src = h * LP + c;
                        m.r = __shfl_sync(0xffffffffu, cur.r, src);
                        m.kb = __shfl_sync(0xffffffffu, cur.kb, src);
                        m.L = __shfl_sync(0xffffffffu, cur.L, src);
                        m.di = __shfl_sync(0xffffffffu, cur.di, src);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) m.bv[v] = __shfl_sync(0xffffffffu, cur.bv[v], src);
                        m.pv = (TX)0;
                        m.pj = 0;
                        if (lane < m.L) {
                            m.pv = ddf_cvt<TX>(A.val[m.kb + lane]);
                            m.pj = A.col[m.kb + lane];
                        }
                        qrow_solve<TV, TX, LY>(m, A.col, A.val, A.X, A.nrhs, lane, A.status, abort_flag, A.cap_ns);
                    }
                }
                cur = nxt;
            }
        }
    }
}

// A warp's ticket, taken by lane 0 and shared with the warp.
__device__ __forceinline__ int64_t take_ticket(uint32_t* ticket, int lane) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1u);
    return (int64_t)__shfl_sync(0xffffffffu, t, 0);
}

// Multi-RHS forward substitution over the level-ordered plan.  A persistent
// grid of warps takes the SpTRSV plan's work units from a ticket, each warp
// on its own, upt consecutive units per ticket (ddf_tune picks upt).  A warp
// holding unit u waits only on rows of units before u, which running warps
// hold or have finished, so the lowest unfinished unit can always proceed
// (no co-residency needed, no cooperative launch).  The next ticket is taken
// before the current units start.
template <typename TV, typename TX, class LY>
__global__ void __launch_bounds__(DDF_CTA_THREADS, SPTRSM_MIN_CTAS) k_sptrsm(SolveArgs<TV, TX> A) {
    const int lane = threadIdx.x & 31;
    int64_t t = take_ticket(A.ticket, lane);
    while (t * A.upt < A.nunits) {
        const int64_t t_next = take_ticket(A.ticket, lane);
        solve_units<TV, TX, LY>(A, t * A.upt, min(t * A.upt + A.upt, A.nunits), lane);
        t = t_next;
    }
}

// A batch's SpMV and SpTRSV in one launch: the tickets first hand out the
// solve's units (as in k_sptrsm), then the SpMV's work items (its three unit
// arrays, then its two tile arrays), one item per ticket.  SpMV items wait on
// nothing, so the argument of k_sptrsm still holds, and warps that find no
// solve unit left run the products while the solve's deep levels finish.
template <typename TV, typename TX, class LY>
__global__ void __launch_bounds__(DDF_CTA_THREADS, SPTRSM_MIN_CTAS)
k_batch(SolveArgs<TV, TX> S, MulArgs<TV, TX> M) {
    const int lane = threadIdx.x & 31;
    const int64_t ts = (S.nunits + S.upt - 1) / S.upt;
    const int64_t c0 = M.nunits[0], c1 = c0 + M.nunits[1], c2 = c1 + M.nunits[2];
    const int64_t c3 = c2 + M.ntiles[0], c4 = c3 + M.ntiles[1];
    int64_t t = take_ticket(S.ticket, lane);
    while (t < ts + c4) {
        const int64_t t_next = take_ticket(S.ticket, lane);
        if (t < ts) {
            solve_units<TV, TX, LY>(S, t * S.upt, min(t * S.upt + S.upt, S.nunits), lane);
        } else {
            const int64_t i = t - ts;
            if (i < c0) spmm_unit<TV, TX, LY>(M, M.units[0][i], lane);
            else if (i < c1) spmm_unit<TV, TX, LY>(M, M.units[1][i - c0], lane);
            else if (i < c2) spmm_unit<TV, TX, LY>(M, M.units[2][i - c1], lane);
            else if (i < c3) spmm_tile<TV, TX, LY>(M, M.tiles[0][i - c2], lane);
            else spmm_tile<TV, TX, LY>(M, M.tiles[1][i - c3], lane);
        }
        t = t_next;
    }
}

// Work items and ticket order of a batch's solve.  In the block-diagonal
// plan, level l holds the rows of every matrix at its own level l, so in
// plain level order the deep matrices' last levels (few rows each, a chain
// of dependency hops) run only after the shallow matrices' wide levels are
// done.  The solve's items are the plan's units split where the matrix
// changes (a codelet may run across the end of one matrix's rows into the
// next one's) and around rows of more than SEG_POINTS points; such a row
// becomes ceil(L / SEG_POINTS) segment items that different warps run at the
// same time (the last one to finish adds the partial sums in segment order).
// The items are sorted by normalized level, l / (depth of their matrix + 1),
// ties in level order, which spreads every matrix over the whole run: the
// deep chains advance beside the wide levels.  The order is topological: an
// item's dependencies are rows of its own matrix at lower levels, whose keys
// are no larger and which come first among equal keys; segments of one row
// never wait on one another.
constexpr int ORDER_KEY_BITS = 20;

__device__ __forceinline__ int32_t last_le(const int32_t* __restrict__ a, int32_t n, int32_t v) {
    int32_t lo = 0, hi = n - 1;   // the last i with a[i] <= v (a[0] <= v)
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (a[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool long_row(const int32_t* __restrict__ st, int64_t q) {
    return st[q + 1] - st[q] > SEG_POINTS;
}

// flag[q] = 1 where a range starts: a unit's first position, a position
// whose row belongs to another matrix than the row before it, a long row,
// or the position after a long row
__global__ void k_range_flags(int32_t n, int64_t nu, const int32_t* __restrict__ unit_q,
                              const int32_t* __restrict__ seq, const int32_t* __restrict__ st,
                              const int32_t* __restrict__ moff, int32_t count, int32_t* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nu) flag[unit_q[i]] = 1;
    if (i >= n) return;
    if (long_row(st, i) || (i > 0 && long_row(st, i - 1))) flag[i] = 1;
    if (i > 0 && last_le(moff, count, seq[i]) != last_le(moff, count, seq[i - 1])) flag[i] = 1;
}

__global__ void k_range_write(int32_t n, const int32_t* __restrict__ flag, const int64_t* __restrict__ off,
                              int32_t* __restrict__ rq) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n && flag[q]) rq[off[q]] = (int32_t)q;
}

// per range: its matrix and level (and the matrix's depth), its items (1, or
// the segments of a long row) and partial-sum slots (0, or one per segment)
__global__ void k_range_level(int64_t nr, const int32_t* __restrict__ rq, const int32_t* __restrict__ seq,
                              const int32_t* __restrict__ st, const int32_t* __restrict__ part_ptr, int32_t depth,
                              const int32_t* __restrict__ moff, int32_t count, int32_t* __restrict__ rmat,
                              int32_t* __restrict__ rlev, int32_t* __restrict__ mdepth, int32_t* __restrict__ nitem,
                              int32_t* __restrict__ nslot) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const int32_t q = rq[r];
    const int32_t m = last_le(moff, count, seq[q]);
    const int32_t l = last_le(part_ptr, depth, q);
    rmat[r] = m;
    rlev[r] = l;
    atomicMax(mdepth + m, l);
    const int32_t L = st[q + 1] - st[q];
    const int32_t S = L > SEG_POINTS ? (L + SEG_POINTS - 1) / SEG_POINTS : 0;   // a long row is a range of its own
    nitem[r] = S > 0 ? S : 1;
    nslot[r] = S;
}

__global__ void k_item_write(int64_t nr, const int32_t* __restrict__ rq, const int32_t* __restrict__ rmat,
                             const int32_t* __restrict__ rlev, const int32_t* __restrict__ mdepth,
                             const int32_t* __restrict__ nslot, const int64_t* __restrict__ ioff,
                             const int64_t* __restrict__ soff, int32_t* __restrict__ iq, int2* __restrict__ iseg,
                             uint32_t* __restrict__ key, int32_t* __restrict__ idx) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const uint32_t k = (uint32_t)(((uint64_t)rlev[r] << ORDER_KEY_BITS) / ((uint64_t)mdepth[rmat[r]] + 1));
    const int32_t S = nslot[r];
    for (int32_t j = 0; j < (S > 0 ? S : 1); ++j) {
        const int64_t i = ioff[r] + j;
        iq[i] = rq[r];
        iseg[i] = S > 0 ? make_int2(j, (int32_t)soff[r]) : make_int2(-1, 0);
        key[i] = k;
        idx[i] = (int32_t)i;
    }
}

}  // namespace

// Builds the solve's items of a batch plan whose matrices start at rows
// moff_h[0 .. count - 1] (host array) and keeps those offsets in the plan.
ddf_status ddf_build_mrhs_items(ddf_plan_s* p, const int32_t* moff_h, int32_t count, cudaStream_t s) {
    const int64_t nu = p->nunits[0];
    const int32_t n = p->n;
    if (nu < 1 || n < 2 || count < 2 || p->nblocks > 0) return DDF_OK;
    int32_t *moff = nullptr, *flag = nullptr, *rq = nullptr, *rmat = nullptr, *rlev = nullptr, *mdepth = nullptr;
    int32_t *nitem = nullptr, *nslot = nullptr, *iq = nullptr, *idx = nullptr;
    int2* iseg = nullptr;
    int64_t *off = nullptr, *ioff = nullptr, *soff = nullptr;
    uint32_t* key = nullptr;
    double* part = nullptr;
    uint32_t* cnt = nullptr;
    int64_t nr = 0, tot[2] = {0, 0};
    ddf_status st = ddf_alloc(&moff, count, s);
    if (!st) st = ddf_alloc(&flag, n, s);
    if (!st) st = ddf_alloc(&off, (int64_t)n + 1, s);
    if (!st && cudaMemcpyAsync(moff, moff_h, sizeof(int32_t) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = DDF_ERR_CUDA;
    if (!st && cudaMemsetAsync(flag, 0, sizeof(int32_t) * n, s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (!st) {
        k_range_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nu, p->unit_q, p->seq, p->starts, moff, count,
                                                                   flag);
        ddf_count_launch();
        if (cudaGetLastError() != cudaSuccess) st = DDF_ERR_CUDA;
    }
    if (!st) st = ddf_scan_i32_to_i64(flag, off, n, s);
    if (!st && (cudaMemcpyAsync(&nr, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess))
        st = DDF_ERR_CUDA;
    if (!st) st = ddf_alloc(&rq, nr, s);
    if (!st) st = ddf_alloc(&rmat, nr, s);
    if (!st) st = ddf_alloc(&rlev, nr, s);
    if (!st) st = ddf_alloc(&nitem, nr, s);
    if (!st) st = ddf_alloc(&nslot, nr, s);
    if (!st) st = ddf_alloc(&ioff, nr + 1, s);
    if (!st) st = ddf_alloc(&soff, nr + 1, s);
    if (!st) st = ddf_alloc(&mdepth, count, s);
    if (!st && cudaMemsetAsync(mdepth, 0, sizeof(int32_t) * count, s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (!st) {
        const unsigned g = (unsigned)((nr + 255) / 256);
        k_range_write<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, flag, off, rq);
        ddf_count_launch();
        k_range_level<<<g, 256, 0, s>>>(nr, rq, p->seq, p->starts, p->part_ptr, p->depth, moff, count, rmat, rlev,
                                       mdepth, nitem, nslot);
        ddf_count_launch();
        if (cudaGetLastError() != cudaSuccess) st = DDF_ERR_CUDA;
    }
    if (!st) st = ddf_scan_i32_to_i64(nitem, ioff, nr, s);
    if (!st) st = ddf_scan_i32_to_i64(nslot, soff, nr, s);
    if (!st && (cudaMemcpyAsync(tot, ioff + nr, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(tot + 1, soff + nr, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess))
        st = DDF_ERR_CUDA;
    const int64_t ni = tot[0], ns = tot[1];
    if (!st) st = ddf_alloc(&iq, ni, s);
    if (!st) st = ddf_alloc(&iseg, ni, s);
    if (!st) st = ddf_alloc(&key, ni, s);
    if (!st) st = ddf_alloc(&idx, ni, s);
    if (!st) st = ddf_alloc(&part, ns * NRHS_MAX, s);
    if (!st) st = ddf_alloc(&cnt, ns, s);
    if (!st && ns > 0 && cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * ns, s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (!st) {
        k_item_write<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(nr, rq, rmat, rlev, mdepth, nslot, ioff, soff, iq,
                                                                   iseg, key, idx);
        ddf_count_launch();
        if (cudaGetLastError() != cudaSuccess) st = DDF_ERR_CUDA;
    }
    if (!st) st = ddf_radix_sort_u32(key, idx, ni, 1u << ORDER_KEY_BITS, s);
    if (!st) {
        p->mrhs_q = iq;
        p->mrhs_seg = iseg;
        p->mrhs_order = idx;
        p->mrhs_nr = ni;
        p->mrhs_part = part;
        p->mrhs_cnt = cnt;
        p->mrhs_ns = ns;
        p->mrhs_moff = moff;
        p->mrhs_nmat = count;
        iq = idx = nullptr;
        iseg = nullptr;
        part = nullptr;
        cnt = nullptr;
        moff = nullptr;
    }
    ddf_free(moff, s);
    ddf_free(flag, s);
    ddf_free(off, s);
    ddf_free(rq, s);
    ddf_free(rmat, s);
    ddf_free(rlev, s);
    ddf_free(nitem, s);
    ddf_free(nslot, s);
    ddf_free(ioff, s);
    ddf_free(soff, s);
    ddf_free(mdepth, s);
    ddf_free(iq, s);
    ddf_free(iseg, s);
    ddf_free(key, s);
    ddf_free(idx, s);
    ddf_free(part, s);
    ddf_free(cnt, s);
    return st;
}

namespace {

unsigned grid_units(int64_t nunits, int sm) {
    int64_t ctas = (nunits + DDF_WARPS_PER_CTA - 1) / DDF_WARPS_PER_CTA;
    int64_t cap = (int64_t)sm * 32;
    return (unsigned)std::max<int64_t>(1, std::min(ctas, cap));
}

// Lanes per row of X for the 16-byte form (nrhs = VEC * LP, LP a power of two
// from 2 to 16, every block 16-byte aligned), else 0 (one element per lane).
template <typename TX>
int vector_lp(int32_t nrhs, std::initializer_list<const void*> blocks) {
    constexpr int VEC = 16 / (int)sizeof(TX);
    if (nrhs % VEC) return 0;
    for (const void* b : blocks)
        if ((uintptr_t)b & 15u) return 0;
    const int lp = nrhs / VEC;
    return (lp == 2 || lp == 4 || lp == 8 || (lp == 16 && VEC == 2)) ? lp : 0;
}

// Calls f with the lane layout for (nrhs, blocks): Lay<TX, VEC, LP> or the
// one-element layout.
template <typename TX, typename F>
void with_layout(int32_t nrhs, std::initializer_list<const void*> blocks, F&& f) {
    constexpr int VEC = 16 / (int)sizeof(TX);
    switch (vector_lp<TX>(nrhs, blocks)) {
        case 2: f(Lay<TX, VEC, 2>{}); break;
        case 4: f(Lay<TX, VEC, 4>{}); break;
        case 8: f(Lay<TX, VEC, 8>{}); break;
        case 16:
            if constexpr (VEC == 2) f(Lay<TX, VEC, 16>{});
            break;
        default: f(Lay<TX, 1, 32>{});
    }
}

template <typename TV, typename TX>
MulArgs<TV, TX> mul_args(const ddf_plan_s* p, const TV* val, const TX* X, TX* Y, int32_t nrhs) {
    MulArgs<TV, TX> A;
    A.cod = p->cod;
    A.st = p->starts;
    A.col = p->col;
    A.val = val;
    A.X = X;
    A.Y = Y;
    A.nrhs = nrhs;
    for (int k = 0; k < 3; ++k) {
        A.units[k] = p->units[k];
        A.nunits[k] = p->nunits[k];
    }
    for (int k = 0; k < 2; ++k) {
        A.tiles[k] = p->tiles[k];
        A.ntiles[k] = p->ntiles[k];
    }
    return A;
}

template <typename TV, typename TX>
SolveArgs<TV, TX> solve_args(const ddf_plan_s* p, const TV* val, const TX* dinv, const TX* B, TX* X,
                             int32_t nrhs) {
    SolveArgs<TV, TX> A;
    A.n = p->n;
    A.upt = p->mrhs_units_per_ticket > 0 ? p->mrhs_units_per_ticket : 1;
    if (p->mrhs_q) {   // a batch: the items and order of ddf_build_mrhs_items
        A.nunits = p->mrhs_nr;
        A.order = p->mrhs_order;
        A.unit_q = p->mrhs_q;
        A.seg = p->mrhs_seg;
        A.part = reinterpret_cast<TX*>(p->mrhs_part);
        A.cnt = p->mrhs_cnt;
    } else {
        A.nunits = p->nunits[0];
        A.order = nullptr;
        A.unit_q = p->unit_q;
        A.seg = nullptr;
        A.part = nullptr;
        A.cnt = nullptr;
    }
    A.seq = p->seq;
    A.st = p->starts;
    A.col = p->col;
    A.val = val;
    A.dinv = dinv;
    A.B = B;
    A.X = X;
    A.nrhs = nrhs;
    A.ticket = p->ticket;
    A.status = p->status;
    A.cap_ns = p->opts.spin_cap_ns;
    return A;
}

template <typename TV, typename TX>
ddf_status launch_spmm(ddf_plan_s* p, const TV* val, const TX* X, TX* Y, int32_t nrhs, cudaStream_t s) {
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    const MulArgs<TV, TX> A = mul_args<TV, TX>(p, val, X, Y, nrhs);
    int launches = 0;
    with_layout<TX>(nrhs, {X, Y}, [&](auto ly) {
        using LY = decltype(ly);
        for (int k = 0; k < 5; ++k) {
            const int64_t count = k < 3 ? A.nunits[k] : A.ntiles[k - 3];
            if (count <= 0) continue;
            k_spmm<TV, TX, LY><<<grid_units(count, sm), DDF_CTA_THREADS, 0, s>>>(A, k);
            ddf_count_launch();
            ++launches;
        }
    });
    p->last_launches = launches;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// Persistent grid of a ticket kernel: its resident CTAs, at most enough for
// `tickets` warps.
template <typename K>
ddf_status ticket_grid(K kern, int64_t tickets, int sm, unsigned* ctas) {
    int per_sm = 0;
    DDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DDF_CTA_THREADS, 0));
    const int64_t want = (tickets + DDF_WARPS_PER_CTA - 1) / DDF_WARPS_PER_CTA;
    *ctas = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm * std::max(per_sm, 1)));
    return DDF_OK;
}

// X := the fill pattern and the plan's ticket and give-up flag := 0.
template <typename TX>
void fill_solve(ddf_plan_s* p, TX* X, int32_t nrhs, cudaStream_t s, int sm) {
    using RBx = RB<TX>;
    const int64_t ne = (int64_t)p->n * nrhs;
    k_fill_m<typename RBx::U><<<ddf_grid(ne > 0 ? ne : 1, 256, (unsigned)sm * 8), 256, 0, s>>>(
        (typename RBx::U*)X, ne, RBx::SENT, p->ticket);
    ddf_count_launch();
}

template <typename TV, typename TX>
ddf_status launch_sptrsm(ddf_plan_s* p, const TV* val, const TX* dinv, const TX* B, TX* X, int32_t nrhs,
                         cudaStream_t s) {
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    fill_solve<TX>(p, X, nrhs, s, sm);
    ddf_status st = DDF_OK;
    if (p->nunits[0] > 0) {
        const SolveArgs<TV, TX> A = solve_args<TV, TX>(p, val, dinv, B, X, nrhs);
        with_layout<TX>(nrhs, {B, X}, [&](auto ly) {
            using LY = decltype(ly);
            unsigned ctas = 1;
            st = ticket_grid(k_sptrsm<TV, TX, LY>, (A.nunits + A.upt - 1) / A.upt, sm, &ctas);
            if (st) return;
            k_sptrsm<TV, TX, LY><<<ctas, DDF_CTA_THREADS, 0, s>>>(A);
            ddf_count_launch();
        });
    }
    if (st) return st;
    p->last_launches = 2;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// Both executors of a batch in one launch (after the solve's fill).
template <typename TV, typename TX>
ddf_status launch_batch(ddf_plan_s* pa, const TV* va, const TX* X, TX* Y, ddf_plan_s* pl, const TV* vl,
                        const TX* dinv, const TX* B, TX* Xs, int32_t nrhs, cudaStream_t s) {
    const int sm = pl->sm_count > 0 ? pl->sm_count : 152;
    fill_solve<TX>(pl, Xs, nrhs, s, sm);
    const SolveArgs<TV, TX> S = solve_args<TV, TX>(pl, vl, dinv, B, Xs, nrhs);
    const MulArgs<TV, TX> M = mul_args<TV, TX>(pa, va, X, Y, nrhs);
    const int64_t tickets = (S.nunits + S.upt - 1) / S.upt + M.nunits[0] + M.nunits[1] + M.nunits[2] +
                            M.ntiles[0] + M.ntiles[1];
    ddf_status st = DDF_OK;
    if (tickets > 0) {
        with_layout<TX>(nrhs, {X, Y, B, Xs}, [&](auto ly) {
            using LY = decltype(ly);
            unsigned ctas = 1;
            st = ticket_grid(k_batch<TV, TX, LY>, tickets, sm, &ctas);
            if (st) return;
            k_batch<TV, TX, LY><<<ctas, DDF_CTA_THREADS, 0, s>>>(S, M);
            ddf_count_launch();
        });
    }
    if (st) return st;
    pa->last_launches = 0;
    pl->last_launches = 2;
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

__global__ void k_fill_f64(double* __restrict__ a, int64_t n, double v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    return na > 0 && nb > 0 && (const char*)a < (const char*)b + nb && (const char*)b < (const char*)a + na;
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
    st = ddf_finish_plan(p, rp, ci, v, s, out);
    if (st || kind != DDF_SPTRSV) return st;
    std::vector<int32_t> moff((size_t)count);
    for (int32_t i = 0, r = 0; i < count; r += mats[i].n_rows, ++i) moff[(size_t)i] = r;
    st = ddf_build_mrhs_items(*out, moff.data(), count, s);
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (st) {
        ddf_plan_destroy(*out);
        *out = nullptr;
    }
    return st;
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
    if (overlaps(B, bytes, X, bytes)) return DDF_ERR_ARG;
    if (p->n == 0) {
        p->last_launches = 0;
        return DDF_OK;
    }
    return run_multi(p, B, X, nrhs, dtype, (cudaStream_t)stream);
}

ddf_status ddf_batch_run(ddf_plan_t pa, const void* X, void* Y, ddf_plan_t pl, const void* B, void* Xs,
                         int32_t nrhs, ddf_dtype dtype, ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_batch_run");
    ddf_status st = check_multi(pa, X, Y, nrhs, dtype);
    if (!st) st = check_multi(pl, B, Xs, nrhs, dtype);
    if (st) return st;
    if (pa->kind != DDF_SPMV || pl->kind != DDF_SPTRSV) return DDF_ERR_WRONG_KIND;
    const size_t es = dtype == DDF_F64 ? 8 : 4;
    const size_t nx = (size_t)pa->n_cols * nrhs * es, ny = (size_t)pa->n * nrhs * es;
    const size_t ns = (size_t)pl->n * nrhs * es;
    // the outputs Y and Xs are written while X, B (and each other) are read
    if (overlaps(Xs, ns, B, ns) || overlaps(Xs, ns, X, nx) || overlaps(Xs, ns, Y, ny) || overlaps(Y, ny, X, nx) ||
        overlaps(Y, ny, B, ns))
        return DDF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == DDF_F64)
        return launch_batch<double, double>(pa, pa->val, (const double*)X, (double*)Y, pl, pl->val, pl->dinv,
                                            (const double*)B, (double*)Xs, nrhs, s);
    return launch_batch<float, float>(pa, (const float*)pa->val_lp, (const float*)X, (float*)Y, pl,
                                      (const float*)pl->val_lp, pl->dinv_lp, (const float*)B, (float*)Xs, nrhs, s);
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
    // SpMV: tile size of the work units; SpTRSV: work units per warp ticket
    const int32_t cand_spmv[] = {64, 128, 256, 512, 1024, 2048};
    const int32_t cand_trsv[] = {1, 2, 4, 8};
    const bool spmv = p->kind == DDF_SPMV;
    const int nc = spmv ? 6 : 4;
    float best = 3.0e38f;
    int32_t pick = spmv ? p->opts.unit_nnz : p->mrhs_units_per_ticket;
    for (int c = 0; c < nc && !st; ++c) {
        if (spmv) {
            p->opts.unit_nnz = cand_spmv[c];
            st = ddf_build_units(p, s);
        } else {
            p->mrhs_units_per_ticket = cand_trsv[c];
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
        p->mrhs_units_per_ticket = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (best_unit_nnz) *best_unit_nnz = pick;
    return st;
}

ddf_status ddf_tune_cost(const ddf_csr* A, ddf_kind kind, ddf_opts* o, ddf_stream_t stream, int32_t* pick) {
    ddf_nvtx_range nvtx_("ddf_tune_cost");
    if (!A || !o || !A->values || (kind != DDF_SPMV && kind != DDF_SPTRSV)) return DDF_ERR_ARG;
    // Eq. 1 weight sets (w_op, w_codelet, w_index): the default byte costs, a
    // cheaper and a dearer codelet, cheaper and dearer offset entries, and
    // the paper's CPU form
    static const int64_t cand[][3] = {{8, 32, 4}, {8, 8, 4}, {8, 128, 4}, {8, 32, 1}, {8, 32, 16}, {1, 3, 1}};
    constexpr int nc = 6;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nin = kind == DDF_SPMV ? A->n_cols : A->n_rows, nout = A->n_rows;
    double *x = nullptr, *y = nullptr;
    ddf_status st = ddf_alloc(&x, std::max<int64_t>(nin, 1), s);
    if (!st) st = ddf_alloc(&y, std::max<int64_t>(nout, 1), s);
    if (!st && nin > 0) {
        k_fill_f64<<<ddf_grid(nin, 256, 4096), 256, 0, s>>>(x, nin, 1.0);
        ddf_count_launch();
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!st && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = DDF_ERR_CUDA;
    float best = 3.0e38f;
    int32_t win = 0;
    for (int c = 0; c < nc && !st; ++c) {
        ddf_opts oc = *o;
        oc.w_op = cand[c][0];
        oc.w_codelet = cand[c][1];
        oc.w_index = cand[c][2];
        ddf_plan_t p = nullptr;
        st = ddf_inspect(A, kind, &oc, stream, &p);
        if (st) break;
        float ms = 3.0e38f;
        for (int rep = 0; rep < 4 && !st; ++rep) {   // a warm-up, then the fastest of three
            cudaEventRecord(e0, s);
            st = kind == DDF_SPMV ? ddf_spmv(p, x, y, stream) : ddf_sptrsv(p, x, y, stream);
            cudaEventRecord(e1, s);
            if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = DDF_ERR_CUDA;
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0 && t < ms) ms = t;
        }
        if (!st && kind == DDF_SPTRSV) st = ddf_get_status(p, stream);
        ddf_plan_destroy(p);
        if (!st && ms < best) {
            best = ms;
            win = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ddf_free(x, s);
    ddf_free(y, s);
    if (st) return st;
    o->w_op = cand[win][0];
    o->w_codelet = cand[win][1];
    o->w_index = cand[win][2];
    if (pick) *pick = win;
    return cudaStreamSynchronize(s) == cudaSuccess ? DDF_OK : DDF_ERR_CUDA;
}

}  // extern "C"
