// SpMV executor y = A x: one kernel per codelet type (Sec. IV-B, Listing 3).
//
// Rows of BLAS / PSC I codelets with at most DDF_TILE_NMAX points run in
// tiles, one lane per row (k_spmv_tile, below).  Every other codelet (PSC II,
// and BLAS / PSC I rows longer than that) runs in work units:
// a warp runs one work unit (rows [i0b, i0e) of one codelet) with v lanes
// per row (v a power of two): lane li of the row group handles the points
// i1 = li, li + v, ...; the row sum is reduced with xor shuffles inside the
// group and written once.  The three kernels differ only in how they form
// the column h(i0, i1):
//   BLAS   h0 + delta*i0 + sigma*i1          no index loads
//   PSC I  h0 + delta*i0 + s[i1]             s loaded once per unit (first row's columns)
//   PSC II col[g(i0, i1)]                    one index per point, row extents from starts
// Values of BLAS / PSC I codelets sit at g0 + gamma*i0 + i1: consecutive rows
// are contiguous, so a row group's loads are coalesced.
//
// The kernels are templated on the value type TV, the vector types TX / TY
// and the accumulator TA: FP64 throughout for ddf_spmv, and FP32 / BF16
// storage with FP32 products and sums for ddf_spmv_lowp.
#include "ddf_internal.cuh"

namespace {

constexpr int SMAX = 4;          // s entries kept in registers per lane (n <= 4 v)
constexpr int SPMV_BATCH = 4;    // points whose loads a lane issues together
// Resident CTAs per SM the kernels are compiled for.  The SpMV is bound by the
// latency of its gathers, not by the FP64 pipe: 6 CTAs (about 40 registers)
// keep more loads in flight than the 4 that 64 registers allow, despite a few
// spilled registers (measured: 14-17% faster on the stencil matrices).
constexpr int SPMV_MIN_CTAS = 6;

// One row of a BLAS / PSC I codelet: lanes li, li + v, ... of its row group.
template <int TYPE, typename TV, typename TX, typename TA>
__device__ __forceinline__ TA row_strided(const TV* __restrict__ val, const TX* __restrict__ x,
                                          const int32_t* __restrict__ col, int32_t n, int32_t v, int32_t li,
                                          int32_t g, int32_t hb, int32_t sigma, int32_t sref, int32_t h0,
                                          const int32_t* sreg) {
    TA acc = 0;
    const TV* vp = val + g;
    if (TYPE == DDF_BLAS) {
#pragma unroll 4
        for (int32_t i1 = li; i1 < n; i1 += v)
            acc += ddf_cvt<TA>(__ldcs(vp + i1)) * ddf_cvt<TA>(__ldg(x + hb + sigma * i1));
    } else if (sreg != nullptr && n <= SMAX * v) {
#pragma unroll
        for (int k = 0; k < SMAX; ++k) {
            int32_t i1 = li + k * v;
            if (i1 < n) acc += ddf_cvt<TA>(__ldcs(vp + i1)) * ddf_cvt<TA>(__ldg(x + hb + sreg[k]));
        }
    } else {
        // offsets and values of SPMV_BATCH points first, then their x gathers,
        // then the products: a batch's loads are in flight together instead of
        // one offset -> x chain at a time
        const int32_t* sp = col + sref;
        for (int32_t b0 = li; b0 < n; b0 += SPMV_BATCH * v) {
            int32_t sj[SPMV_BATCH];
            TV vv[SPMV_BATCH];
            TX xv[SPMV_BATCH];
#pragma unroll
            for (int k = 0; k < SPMV_BATCH; ++k) {
                const int32_t i1 = b0 + k * v;
                sj[k] = i1 < n ? __ldg(sp + i1) - h0 : 0;
                vv[k] = i1 < n ? __ldcs(vp + i1) : (TV)0;
            }
#pragma unroll
            for (int k = 0; k < SPMV_BATCH; ++k) xv[k] = (b0 + k * v < n) ? __ldg(x + hb + sj[k]) : (TX)0;
#pragma unroll
            for (int k = 0; k < SPMV_BATCH; ++k) acc += ddf_cvt<TA>(vv[k]) * ddf_cvt<TA>(xv[k]);
        }
    }
    return acc;
}

template <typename TY, typename TA>
__device__ __forceinline__ TY store_cvt(TA v) { return (TY)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 store_cvt<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

template <int TYPE, typename TV, typename TX, typename TY, typename TA>
__global__ void __launch_bounds__(DDF_CTA_THREADS, SPMV_MIN_CTAS)
k_spmv(const dcod* __restrict__ cod, const dunit* __restrict__ units, int64_t nunits,
       const int32_t* __restrict__ st, const int32_t* __restrict__ col, const TV* __restrict__ val,
       const TX* __restrict__ x, TY* __restrict__ y) {
    __shared__ int8_t rowslot[DDF_WARPS_PER_CTA][256];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += nw) {
        const dunit U = units[u];
        const int v = U.v;
        const int lg = __ffs(v) - 1;
        const int rpw = 32 >> lg;
        const int sub = lane >> lg;
        const int li = lane & (v - 1);
        if (TYPE != DDF_PSC2 && U.i0b < 0) {
            // group of -U.i0b small codelets with U.i0e rows in total: lane k holds
            // codelet k's descriptor, rowslot maps a unit row to its codelet
            const int cnt = -U.i0b;
            dcod C;
            int32_t m = 0;
            if (lane < cnt) {
                C = cod[U.cod + lane];
                m = C.m;
            } else {
                C = cod[U.cod];
            }
            int32_t incl = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int32_t excl = incl - m;
            __syncwarp();
            for (int32_t r = excl; r < incl; ++r) rowslot[wl][r] = (int8_t)lane;
            __syncwarp();
            const int32_t n = C.n;   // equal for every codelet of the group (lane 0's is used)
            const int32_t n0 = __shfl_sync(0xffffffffu, n, 0);
            for (int32_t kb = 0; kb < U.i0e; kb += rpw) {
                const int32_t k = kb + sub;
                const bool act = k < U.i0e;
                const int slot = act ? rowslot[wl][k] : 0;
                const int32_t i0 = k - __shfl_sync(0xffffffffu, excl, slot);
                const int32_t f0 = __shfl_sync(0xffffffffu, C.f0, slot);
                const int32_t rho = __shfl_sync(0xffffffffu, C.rho, slot);
                const int32_t g0 = __shfl_sync(0xffffffffu, C.g0, slot);
                const int32_t gamma = __shfl_sync(0xffffffffu, C.gamma, slot);
                const int32_t h0 = __shfl_sync(0xffffffffu, C.h0, slot);
                const int32_t delta = __shfl_sync(0xffffffffu, C.delta, slot);
                const int32_t sigma = __shfl_sync(0xffffffffu, C.sigma, slot);
                const int32_t sref = __shfl_sync(0xffffffffu, C.sref, slot);
                TA acc = 0;
                if (act)
                    acc = row_strided<TYPE, TV, TX, TA>(val, x, col, n0, v, li, g0 + gamma * i0, h0 + delta * i0,
                                                        sigma, sref, h0, nullptr);
                for (int o = v >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (act && li == 0) y[f0 + rho * i0] = store_cvt<TY, TA>(acc);
            }
            __syncwarp();
            continue;
        }
        const dcod C = cod[U.cod];
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
            TA acc = 0;
            int32_t r = 0;
            if (act) {
                r = C.f0 + C.rho * i0;
                if (TYPE == DDF_PSC2) {
                    const int32_t q = C.q0 + i0;
                    const int32_t kb = st[q], ke = st[q + 1];
#pragma unroll 4
                    for (int32_t k = kb + li; k < ke; k += v)
                        acc += ddf_cvt<TA>(__ldcs(val + k)) * ddf_cvt<TA>(__ldg(x + __ldcs(col + k)));
                } else {
                    acc = row_strided<TYPE, TV, TX, TA>(val, x, col, C.n, v, li, C.g0 + C.gamma * i0,
                                                        C.h0 + C.delta * i0, C.sigma, C.sref, C.h0, sreg);
                }
            }
            for (int o = v >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (act && li == 0) y[r] = store_cvt<TY, TA>(acc);
        }
    }
}

// Tiled rows (runs of BLAS / PSC I codelets with short rows): one lane per
// row, no reduction.  A warp takes TILES_PER_WARP consecutive tiles of
// DDF_TILE_ROWS rows; lane l runs row r = l % DDF_TILE_ROWS of tile
// l / DDF_TILE_ROWS.  The tile's values are point-major, so for each point i1
// the lanes of a tile read one contiguous stretch of w values; the column of
// point i1 is h0 + delta*i0 + sigma*i1 (BLAS) or col[sref + i1] + delta*i0
// (PSC I: s[i1] + h0 is the codelet's first row's column, read by every lane
// of the codelet from the same address).  Each lane issues the loads of
// TILE_BATCH points before using any, then one fused multiply-add per point.
constexpr int TILES_PER_WARP = 32 / DDF_TILE_ROWS;
constexpr int TILE_BATCH = 4;

template <int TYPE, typename TV, typename TX, typename TY, typename TA>
__global__ void __launch_bounds__(DDF_CTA_THREADS, SPMV_MIN_CTAS)
k_spmv_tile(const dcod* __restrict__ cod, const dtile* __restrict__ tiles, int64_t ntiles,
            const int32_t* __restrict__ col, const TV* __restrict__ val, const TX* __restrict__ x,
            TY* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int sub = lane / DDF_TILE_ROWS, r = lane % DDF_TILE_ROWS;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tb = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * TILES_PER_WARP; tb < ntiles;
         tb += nw * TILES_PER_WARP) {
        const int64_t t = tb + sub;
        int32_t n = 0, w = 0, fr = 0;
        const TV* vp = val;
        const int32_t* sp = col;   // PSC I: the codelet's s (its first row's columns)
        int32_t hb = 0, sg = 0;    // BLAS: column h0 + delta*i0 + sigma*i1; PSC I: col[sref + i1] + hb
        if (t < ntiles) {
            const dtile T = tiles[t];
            w = (int32_t)(T.meta & 7u) + 1;
            if (r < w) {
                const dcod C = cod[T.cod + (int32_t)((T.meta >> (3 + 3 * r)) & 7u)];
                const int32_t i0 = T.q + r - C.q0;
                n = C.n;
                fr = C.f0 + C.rho * i0;
                vp = val + T.vb + r;
                if (TYPE == DDF_BLAS) {
                    hb = C.h0 + C.delta * i0;
                    sg = C.sigma;
                } else {
                    sp = col + C.sref;
                    hb = C.delta * i0;
                }
            }
        }
        TA acc = 0;
        int32_t i1 = 0;
        for (; i1 + TILE_BATCH <= n; i1 += TILE_BATCH) {
            TV vv[TILE_BATCH];
            int32_t jj[TILE_BATCH];
            TX xv[TILE_BATCH];
#pragma unroll
            for (int k = 0; k < TILE_BATCH; ++k) {
                jj[k] = TYPE == DDF_BLAS ? hb + sg * (i1 + k) : __ldg(sp + i1 + k) + hb;
                vv[k] = __ldcs(vp + (int64_t)(i1 + k) * w);
            }
#pragma unroll
            for (int k = 0; k < TILE_BATCH; ++k) xv[k] = __ldg(x + jj[k]);
#pragma unroll
            for (int k = 0; k < TILE_BATCH; ++k) acc += ddf_cvt<TA>(vv[k]) * ddf_cvt<TA>(xv[k]);
        }
        for (; i1 < n; ++i1) {
            const int32_t j = TYPE == DDF_BLAS ? hb + sg * i1 : __ldg(sp + i1) + hb;
            acc += ddf_cvt<TA>(__ldcs(vp + (int64_t)i1 * w)) * ddf_cvt<TA>(__ldg(x + j));
        }
        if (r < w) y[fr] = store_cvt<TY, TA>(acc);
    }
}

// PSC II units (whole consecutive rows, at most unit_nnz points).  Lane l
// takes the unit's points [l K, (l + 1) K), K = ceil(points / 32), and adds
// their products with fused multiply-adds in point order, row by row: a row
// that starts and ends inside the lane's stretch is written at once.  A row
// that crosses stretch boundaries has a partial sum in each lane it touches;
// a 5-step scan over the lanes carries each lane's last partial into the
// lanes that continue the same row, and the lane where the row ends writes
// it.  About K + 7 FP64 warp instructions per unit (K fused multiply-adds, the
// scan's adds), and no lane waits on a long row while the others idle.  The
// unit's row starts are staged in shared memory for the lanes to find their
// rows.  Empty rows are written 0 by a separate pass over the rows.  Units of
// more than PSC2_STAGE points (one row each, since a unit closes before a row
// that would take it past unit_nnz) run the row with all 32 lanes and one
// shuffle reduction; rows of more than DDF_LONG_ROW points run one CTA per
// row: the first nlong CTAs of the launch take one such row each (threads
// over the row's points, then a reduction in a fixed order: shuffles inside
// each warp, warps in index order), and the other CTAs walk the units,
// skipping those rows.  Every sum has a fixed order, so results do not
// depend on scheduling.
constexpr int PSC2_STAGE = 256;   // most points of a unit run by the lane stretches
constexpr int PSC2_ROWS = 256;    // rows of a unit (the unit builder's limit)

template <typename TV, typename TX, typename TY, typename TA>
__global__ void __launch_bounds__(DDF_CTA_THREADS, SPMV_MIN_CTAS)
k_spmv_psc2(const dcod* __restrict__ cod, const dunit* __restrict__ units, int64_t nunits,
            const int32_t* __restrict__ long_q, int64_t nlong, const int32_t* __restrict__ st,
            const int32_t* __restrict__ col, const TV* __restrict__ val, const TX* __restrict__ x,
            TY* __restrict__ y) {
    __shared__ int32_t srow_all[DDF_WARPS_PER_CTA][PSC2_ROWS + 1];
    __shared__ TA part[DDF_WARPS_PER_CTA];
    const int lane = threadIdx.x & 31;
    if ((int64_t)blockIdx.x < nlong) {
        const int32_t q = long_q[blockIdx.x];
        const int32_t a = st[q], b = st[q + 1];
        TA acc = 0;
#pragma unroll 4
        for (int32_t k = a + (int32_t)threadIdx.x; k < b; k += DDF_CTA_THREADS)
            acc += ddf_cvt<TA>(__ldcs(val + k)) * ddf_cvt<TA>(__ldg(x + __ldcs(col + k)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            TA t = 0;
#pragma unroll
            for (int w = 0; w < DDF_WARPS_PER_CTA; ++w) t += part[w];
            y[q] = store_cvt<TY, TA>(t);   // SpMV positions are the rows
        }
        return;
    }
    int32_t* srow = srow_all[threadIdx.x >> 5];
    const int64_t nw = ((int64_t)(gridDim.x - nlong) * blockDim.x) >> 5;
    for (int64_t u = (((int64_t)blockIdx.x - nlong) * blockDim.x + threadIdx.x) >> 5; u < nunits; u += nw) {
        const dunit U = units[u];
        const dcod C = cod[U.cod];
        const int32_t qa = C.q0 + U.i0b, qb = C.q0 + U.i0e;
        const int32_t ka = st[qa], kb = st[qb];
        const int32_t T = kb - ka;
        const int32_t fb = C.f0 + C.rho * U.i0b;   // y index of the unit's first row
        if (T > PSC2_STAGE) {
            if (T > DDF_LONG_ROW) continue;   // one of the CTAs above
            TA acc = 0;
#pragma unroll 4
            for (int32_t k = ka + lane; k < kb; k += 32)
                acc += ddf_cvt<TA>(__ldcs(val + k)) * ddf_cvt<TA>(__ldg(x + __ldcs(col + k)));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) y[fb] = store_cvt<TY, TA>(acc);
            continue;
        }
        const int32_t R = qb - qa;
        for (int32_t i = lane; i <= R; i += 32) srow[i] = st[qa + i] - ka;
        __syncwarp();
        // empty rows
        for (int32_t i = lane; i < R; i += 32)
            if (srow[i + 1] == srow[i]) y[fb + C.rho * i] = store_cvt<TY, TA>((TA)0);
        const int32_t K = (T + 31) >> 5;
        const int32_t e0 = min(lane * K, T), e1 = min(e0 + K, T);
        TA hp = 0, tp = 0;
        int32_t hr = 0, tr = 0;
        bool cont = false, single = true;
        if (e0 < e1) {
            // the row holding point e0: the last row starting at or before it
            int32_t lo = 0, hi = R - 1;
            while (lo < hi) {
                const int32_t mid = (lo + hi + 1) >> 1;
                if (srow[mid] <= e0) lo = mid;
                else hi = mid - 1;
            }
            int32_t r = lo;
            hr = r;
            cont = srow[r] < e0;
            TA acc = 0;
            int32_t next = srow[r + 1];
            for (int32_t eb = e0; eb < e1; eb += 4) {
                // four points' loads in flight together, then their multiply-adds in point order
                TA pa[4], px[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    pa[i] = px[i] = (TA)0;
                    if (eb + i < e1) {
                        pa[i] = ddf_cvt<TA>(__ldcs(val + ka + eb + i));
                        px[i] = ddf_cvt<TA>(__ldg(x + __ldcs(col + ka + eb + i)));
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int32_t e = eb + i;
                    if (e >= e1) break;
                    while (next <= e) {   // row r ended before point e
                        if (single) hp = acc;
                        else if (next > srow[r]) y[fb + C.rho * r] = store_cvt<TY, TA>(acc);   // inside the stretch
                        single = false;
                        acc = 0;
                        ++r;
                        next = srow[r + 1];
                    }
                    acc += pa[i] * px[i];
                }
            }
            tr = r;
            tp = acc;
            if (single) hp = acc;
        }
        // carry_out(l) = tp(l) + [single(l) and cont(l)] carry_out(l - 1): a scan over the lanes
        TA cb = tp;
        bool ca = single && cont && e0 < e1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const TA pb = __shfl_up_sync(0xffffffffu, cb, o);
            const bool pa = __shfl_up_sync(0xffffffffu, ca, o);
            if (lane >= o) {
                if (ca) cb += pb;
                ca = ca && pa;
            }
        }
        const TA prev = __shfl_up_sync(0xffffffffu, cb, 1);
        const TA cin = (lane > 0 && cont) ? prev : (TA)0;
        if (e0 < e1) {
            if (!single) {
                y[fb + C.rho * hr] = store_cvt<TY, TA>(hp + cin);   // the head row ended in the stretch
                if (srow[tr + 1] == e1) y[fb + C.rho * tr] = store_cvt<TY, TA>(tp);
            } else if (srow[hr + 1] == e1) {
                y[fb + C.rho * hr] = store_cvt<TY, TA>(hp + cin);
            }
        }
        __syncwarp();
    }
}

unsigned grid_for(int64_t nunits, int sm_count) {
    int64_t ctas = (nunits + DDF_WARPS_PER_CTA - 1) / DDF_WARPS_PER_CTA;
    int64_t cap = (int64_t)sm_count * 32;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    return (unsigned)ctas;
}

template <typename TV, typename TX, typename TY, typename TA>
int launch_all(ddf_plan_s* p, const TV* val, const TX* x, TY* y, cudaStream_t s) {
    int launches = 0;
    int sm = p->sm_count > 0 ? p->sm_count : 152;
    if (p->ntiles[DDF_BLAS] > 0) {
        k_spmv_tile<DDF_BLAS, TV, TX, TY, TA>
            <<<grid_for((p->ntiles[0] + TILES_PER_WARP - 1) / TILES_PER_WARP, sm), DDF_CTA_THREADS, 0, s>>>(
                p->cod, p->tiles[0], p->ntiles[0], p->col, val, x, y);
        ddf_count_launch();
        ++launches;
    }
    if (p->ntiles[DDF_PSC1] > 0) {
        k_spmv_tile<DDF_PSC1, TV, TX, TY, TA>
            <<<grid_for((p->ntiles[1] + TILES_PER_WARP - 1) / TILES_PER_WARP, sm), DDF_CTA_THREADS, 0, s>>>(
                p->cod, p->tiles[1], p->ntiles[1], p->col, val, x, y);
        ddf_count_launch();
        ++launches;
    }
    if (p->nunits[DDF_BLAS] > 0) {
        k_spmv<DDF_BLAS, TV, TX, TY, TA><<<grid_for(p->nunits[0], sm), DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->units[0], p->nunits[0], p->starts, p->col, val, x, y);
        ddf_count_launch();
        ++launches;
    }
    if (p->nunits[DDF_PSC1] > 0) {
        k_spmv<DDF_PSC1, TV, TX, TY, TA><<<grid_for(p->nunits[1], sm), DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->units[1], p->nunits[1], p->starts, p->col, val, x, y);
        ddf_count_launch();
        ++launches;
    }
    if (p->nunits[DDF_PSC2] > 0) {
        // the long rows' CTAs first, then those walking the units
        const int64_t ctas = (int64_t)grid_for(p->nunits[2], sm) + p->nlong;
        k_spmv_psc2<TV, TX, TY, TA><<<(unsigned)ctas, DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->units[2], p->nunits[2], p->long_q, p->nlong, p->starts, p->col, val, x, y);
        ddf_count_launch();
        ++launches;
    }
    return launches;
}

}  // namespace

ddf_status ddf_launch_spmv(ddf_plan_s* p, const double* x, double* y, cudaStream_t s) {
    p->last_launches = launch_all<double, double, double, double>(p, p->val, x, y, s);
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

ddf_status ddf_launch_spmv_lp(ddf_plan_s* p, const void* x, void* y, int vec_dtype, cudaStream_t s) {
    using bf = __nv_bfloat16;
    int l = 0;
    if (p->vdtype == DDF_F32 && vec_dtype == DDF_F32)
        l = launch_all<float, float, float, float>(p, (const float*)p->val_lp, (const float*)x, (float*)y, s);
    else if (p->vdtype == DDF_F32 && vec_dtype == DDF_BF16)
        l = launch_all<float, bf, bf, float>(p, (const float*)p->val_lp, (const bf*)x, (bf*)y, s);
    else if (p->vdtype == DDF_BF16 && vec_dtype == DDF_F32)
        l = launch_all<bf, float, float, float>(p, (const bf*)p->val_lp, (const float*)x, (float*)y, s);
    else if (p->vdtype == DDF_BF16 && vec_dtype == DDF_BF16)
        l = launch_all<bf, bf, bf, float>(p, (const bf*)p->val_lp, (const bf*)x, (bf*)y, s);
    else
        return DDF_ERR_ARG;
    p->last_launches = l;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}
