// Plan validation: every index an executor derives from a plan is recomputed
// from the codelet descriptors and the work units, the same way the executors
// compute it, and checked against the sizes of the arrays it addresses:
//   rows           f(i0) = f0 + rho*i0 (SpMV, and strided f) or seq[q]
//   value extents  g: starts[q] .. starts[q+1] (PSC II) or g0 + gamma*i0, n points
//   columns        h: h0 + delta*i0 + sigma*i1 (BLAS), h0 + delta*i0 + s[i1] (PSC I),
//                     col[g] (PSC II), inside [0, n_cols)
//   value tiles    (SpMV) runs of codelets of one type and row length, and
//                  tiles whose rows lie in the codelets they name
// and, for SpTRSV, that every column names a row solved before the row that
// reads it: below the diagonal and in an earlier partition.  Work units must
// name codelets and row ranges that exist.  ddf_plan_load runs this on every
// plan it rebuilds, so that a buffer whose checksum matches but whose content
// was altered cannot make an executor read or write outside its arrays.
#include <algorithm>

#include "ddf_internal.cuh"

namespace {

__device__ __forceinline__ void fail(int32_t* err, ddf_status code) { atomicMin(err, (int)code); }

// pos[row] = position of the row in the plan's sequence (SpTRSV).
__global__ void k_pos_of(int32_t n, const int32_t* __restrict__ seq, int32_t* __restrict__ pos,
                         int32_t* __restrict__ err) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int32_t r = seq[q];
    if (r < 0 || r >= n) {
        fail(err, DDF_ERR_OUT_OF_RANGE);
        return;
    }
    pos[r] = (int32_t)q;
}

// One thread per codelet.
__global__ void k_check_codelets(int kind, int64_t ncod, const dcod* __restrict__ cod, int32_t n, int32_t n_cols,
                                 int64_t npts, int32_t depth, const int32_t* __restrict__ part_ptr,
                                 const int32_t* __restrict__ seq, const int32_t* __restrict__ st,
                                 const int32_t* __restrict__ col, const int32_t* __restrict__ pos,
                                 int32_t* __restrict__ err) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncod) return;
    const dcod C = cod[c];
    if (C.type < 0 || C.type > 2 || C.m < 1 || C.q0 < 0 || (int64_t)C.q0 + C.m > n || C.part < 0 ||
        C.part >= depth || C.q0 < part_ptr[C.part] || (int64_t)C.q0 + C.m > part_ptr[C.part + 1] ||
        (C.type != DDF_PSC2 && C.n < 0)) {
        fail(err, DDF_ERR_ARG);
        return;
    }
    const bool trsv = kind == DDF_SPTRSV;
    if (C.flags & DC_TILED) {
        // a run of SpMV value tiles: consecutive codelets of one type and row
        // length, every row of length n (the tiles' values are w x n blocks)
        bool ok = !trsv && C.type != DDF_PSC2 && C.n >= 0 && C.n <= DDF_TILE_NMAX && C.pad0 >= 0 &&
                  C.pad0 <= C.q0 && (int64_t)C.q0 + C.m <= C.pad1 && C.pad1 <= n;
        if (ok && C.q0 > C.pad0) {
            const dcod P = cod[c > 0 ? c - 1 : 0];
            ok = c > 0 && (P.flags & DC_TILED) && P.type == C.type && P.n == C.n && P.pad0 == C.pad0 &&
                 P.pad1 == C.pad1 && P.q0 + P.m == C.q0;
        }
        if (ok && C.q0 + C.m < C.pad1) {
            const dcod N = cod[c + 1 < ncod ? c + 1 : c];
            ok = c + 1 < ncod && (N.flags & DC_TILED) && N.type == C.type && N.n == C.n && N.pad0 == C.pad0 &&
                 N.pad1 == C.pad1 && N.q0 == C.q0 + C.m;
        }
        for (int32_t i0 = 0; ok && i0 < C.m; ++i0) ok = st[C.q0 + i0 + 1] - st[C.q0 + i0] == C.n;
        if (!ok) {
            fail(err, DDF_ERR_ARG);
            return;
        }
    }
    const int32_t pstart = part_ptr[C.part];
    for (int32_t i0 = 0; i0 < C.m; ++i0) {
        const int32_t q = C.q0 + i0;
        const int64_t r = (!trsv || (C.flags & DC_F_STRIDED)) ? (int64_t)C.f0 + (int64_t)C.rho * i0
                                                             : (int64_t)seq[q];
        if (r < 0 || r >= n) {
            fail(err, DDF_ERR_OUT_OF_RANGE);
            return;
        }
        int64_t kb, L;
        if (C.type == DDF_PSC2) {
            kb = st[q];
            L = (int64_t)st[q + 1] - kb;
        } else {
            kb = (int64_t)C.g0 + (int64_t)C.gamma * i0;
            L = C.n;
        }
        if (kb < 0 || L < 0 || kb + L > npts || (C.type == DDF_PSC1 && L > 0 && (C.sref < 0 || C.sref + L > npts))) {
            fail(err, DDF_ERR_OUT_OF_RANGE);
            return;
        }
        const int64_t hb = (int64_t)C.h0 + (int64_t)C.delta * i0;
        for (int64_t i1 = 0; i1 < L; ++i1) {
            const int64_t j = C.type == DDF_BLAS   ? hb + (int64_t)C.sigma * i1
                              : C.type == DDF_PSC1 ? hb + ((int64_t)col[C.sref + i1] - C.h0)
                                                   : (int64_t)col[kb + i1];
            if (j < 0 || j >= n_cols) {
                fail(err, DDF_ERR_OUT_OF_RANGE);
                return;
            }
            if (trsv && (j >= r || pos[j] >= pstart)) {
                fail(err, DDF_ERR_NOT_LOWER);
                return;
            }
        }
    }
}

// One thread per work unit.  SpTRSV units are row ranges of one codelet, in
// partition order (a unit never waits on a row that a later unit solves).
__global__ void k_check_units(int kind, int64_t ncod, const dcod* __restrict__ cod, const dunit* __restrict__ units,
                              int64_t nunits, int32_t* __restrict__ err) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nunits) return;
    const dunit U = units[u];
    if (U.v < 1 || U.v > 32 || (U.v & (U.v - 1)) != 0 || U.cod < 0 || U.cod >= ncod) {
        fail(err, DDF_ERR_ARG);
        return;
    }
    if (kind == DDF_SPTRSV) {
        const int32_t pu = units[u - (u > 0)].cod;
        if (U.i0b < 0 || (pu >= 0 && pu < ncod && cod[pu].part > cod[U.cod].part)) {
            fail(err, DDF_ERR_ARG);
            return;
        }
    }
    if (U.i0b >= 0) {
        if (U.i0e <= U.i0b || U.i0e > cod[U.cod].m) fail(err, DDF_ERR_ARG);
        return;
    }
    // a group of -i0b consecutive codelets with i0e rows in all (at most one
    // per lane, at most 256 rows: the executor's per-warp row table)
    const int32_t cnt = -U.i0b;
    if (cnt < 1 || cnt > 32 || (int64_t)U.cod + cnt > ncod) {
        fail(err, DDF_ERR_ARG);
        return;
    }
    // one type (not PSC II) and one row length: the executor reads n from the
    // group's first codelet
    const dcod C0 = cod[U.cod];
    int64_t rows = 0;
    bool same = C0.type != DDF_PSC2;
    for (int32_t k = 0; k < cnt; ++k) {
        const dcod& C = cod[U.cod + k];
        rows += C.m;
        same = same && C.type == C0.type && C.n == C0.n;
    }
    if (!same || rows != U.i0e || rows > 256) fail(err, DDF_ERR_ARG);
}

// One thread per SpMV value tile: rows inside the plan and inside the codelets
// the tile names (tiled, of the list's type and one row length), values from
// the first row's offset.
__global__ void k_check_tiles(int type, int64_t ncod, const dcod* __restrict__ cod, const dtile* __restrict__ tiles,
                              int64_t ntiles, int32_t n, const int32_t* __restrict__ st, int32_t* __restrict__ err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const dtile T = tiles[t];
    const int32_t w = (int32_t)(T.meta & 7u) + 1;
    if (T.cod < 0 || T.cod >= ncod || T.q < 0 || (int64_t)T.q + w > n || T.vb != st[T.q] || (T.meta >> 27) != 0) {
        fail(err, DDF_ERR_ARG);
        return;
    }
    const int32_t n0 = cod[T.cod].n;
    for (int32_t r = 0; r < w; ++r) {
        const int64_t c = (int64_t)T.cod + ((T.meta >> (3 + 3 * r)) & 7u);
        if (c >= ncod) {
            fail(err, DDF_ERR_ARG);
            return;
        }
        const dcod C = cod[c];
        if (!(C.flags & DC_TILED) || C.type != type || C.n != n0 || T.q + r < C.q0 || T.q + r >= C.q0 + C.m) {
            fail(err, DDF_ERR_ARG);
            return;
        }
    }
}

// starts[] of every plan: 0 at the first position, never decreasing, inside
// the point arrays (every executor reads a position's points through it).
__global__ void k_check_starts(int32_t n, int64_t npts, const int32_t* __restrict__ st, int32_t* __restrict__ err) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0 && (st[0] != 0 || (int64_t)st[n] > npts)) fail(err, DDF_ERR_OUT_OF_RANGE);
    if (q < n && st[q + 1] < st[q]) fail(err, DDF_ERR_OUT_OF_RANGE);
}

// SpTRSV: the inspected matrix's rows, kept for ddf_update_values, against
// the plan's layout: position q holds row r = seq[q], whose entries
// orig_rowptr[r] .. re[r] (re = orig_rowptr + 1, or orig_rowend) end with the
// diagonal and fill starts[q] .. starts[q + 1] without it.
__global__ void k_check_rows(int32_t n, int64_t nnz_in, const int32_t* __restrict__ seq,
                             const int32_t* __restrict__ st, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ re, int32_t* __restrict__ err) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int32_t r = seq[q];
    if (r < 0 || r >= n) {
        fail(err, DDF_ERR_OUT_OF_RANGE);
        return;
    }
    const int32_t a = rp[r], e = re[r], b = rp[r + 1];
    if (a < 0 || e <= a || e > b || (int64_t)b > nnz_in || (int64_t)e - a - 1 != (int64_t)st[q + 1] - st[q])
        fail(err, DDF_ERR_OUT_OF_RANGE);
}

__device__ __forceinline__ bool lanes_ok(int32_t v) { return v >= 1 && v <= 32 && (v & (v - 1)) == 0; }

// Coarsened SpTRSV plans: block and chunk tables, and every row of a block's
// positions inside the block (the solve keeps the block's x at r - base).
__global__ void k_check_chunks(int32_t n, int32_t R, int32_t nblocks, int64_t nchunks,
                               const int32_t* __restrict__ blk_chunk, const int32_t* __restrict__ chunk_q0,
                               const int32_t* __restrict__ chunk_meta, const int32_t* __restrict__ seq,
                               const int32_t* __restrict__ st, const int32_t* __restrict__ esplit,
                               int32_t* __restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (blk_chunk[0] != 0 || blk_chunk[nblocks] != nchunks || chunk_q0[0] != 0 || chunk_q0[nchunks] != n))
        fail(err, DDF_ERR_ARG);
    if (i < nblocks) {
        const int32_t c0 = blk_chunk[i], c1 = blk_chunk[i + 1];
        if (c1 < c0 || c0 < 0 || c1 > nchunks) {
            fail(err, DDF_ERR_ARG);
        } else {
            const int64_t base = (int64_t)i * R;
            for (int32_t q = max(chunk_q0[c0], 0); q < chunk_q0[c1] && q < n; ++q)
                if (seq[q] < base || seq[q] >= base + R) {
                    fail(err, DDF_ERR_ARG);
                    break;
                }
        }
    }
    if (i < nchunks) {
        const int32_t a = chunk_q0[i], b = chunk_q0[i + 1], m = chunk_meta[i];
        if (b <= a || a < 0 || b > n || (b - a > DDF_BLK_ROWS_CAP) || !lanes_ok(DDF_CK_VCHAIN(m)) ||
            !lanes_ok(DDF_CK_VPROD(m))) {
            fail(err, DDF_ERR_ARG);
            return;
        }
        const bool direct = (m & DDF_CK_DIRECT) != 0;
        if ((direct && b - a != 1) || (!direct && (int64_t)st[b] - st[a] > DDF_BLK_ENT_CAP)) fail(err, DDF_ERR_ARG);
    }
    if (i < n && (esplit[i] < 0 || esplit[i] > st[i + 1] - st[i])) fail(err, DDF_ERR_ARG);
}

}  // namespace

extern "C" {

ddf_status ddf_plan_validate(ddf_plan_t p) {
    ddf_nvtx_range nvtx_("ddf_plan_validate");
    if (!p) return DDF_ERR_ARG;
    cudaStream_t s = p->stream;
    const int32_t n = p->n;
    const bool trsv = p->kind == DDF_SPTRSV;
    const int64_t npts = trsv ? p->npts : p->nnz;
    int32_t* err = nullptr;
    int32_t* pos = nullptr;
    ddf_status st = ddf_alloc(&err, 1, s);
    if (!st && trsv) st = ddf_alloc(&pos, n, s);
    if (st) {
        ddf_free(err, s);
        return st;
    }
    const int32_t ok = 0x7fffffff;
    ddf_status res = DDF_OK;
    do {
        if (cudaMemcpyAsync(err, &ok, sizeof(ok), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            res = DDF_ERR_CUDA;
            break;
        }
        if (trsv && n > 0) {
            if (cudaMemsetAsync(pos, 0x7f, (size_t)n * sizeof(int32_t), s) != cudaSuccess) {
                res = DDF_ERR_CUDA;
                break;
            }
            k_pos_of<<<ddf_grid(n, 256), 256, 0, s>>>(n, p->seq, pos, err);
            ddf_count_launch();
        }
        if (p->ncod > 0) {
            k_check_codelets<<<ddf_grid(p->ncod, 128), 128, 0, s>>>(p->kind, p->ncod, p->cod, n, p->n_cols, npts,
                                                                    p->depth, p->part_ptr, p->seq, p->starts, p->col,
                                                                    pos, err);
            ddf_count_launch();
        }
        for (int t = 0; t < 3; ++t) {
            if (p->nunits[t] <= 0) continue;
            k_check_units<<<ddf_grid(p->nunits[t], 256), 256, 0, s>>>(p->kind, p->ncod, p->cod, p->units[t],
                                                                      p->nunits[t], err);
            ddf_count_launch();
        }
        for (int t = 0; t < 2; ++t) {
            if (trsv || p->ntiles[t] <= 0) continue;
            k_check_tiles<<<ddf_grid(p->ntiles[t], 256), 256, 0, s>>>(t, p->ncod, p->cod, p->tiles[t],
                                                                      p->ntiles[t], n, p->starts, err);
            ddf_count_launch();
        }
        if (n > 0) {
            k_check_starts<<<ddf_grid((int64_t)n + 1, 256), 256, 0, s>>>(n, npts, p->starts, err);
            ddf_count_launch();
        }
        if (trsv && n > 0 && p->orig_rowptr) {
            const int32_t* re = p->orig_rowend ? p->orig_rowend : p->orig_rowptr + 1;
            k_check_rows<<<ddf_grid(n, 256), 256, 0, s>>>(n, p->nnz, p->seq, p->starts, p->orig_rowptr, re, err);
            ddf_count_launch();
        }
        if (trsv && n > 0 && p->nblocks > 0) {
            const int64_t work = std::max<int64_t>(std::max<int64_t>(p->nblocks, p->nchunks), n) + 1;
            k_check_chunks<<<ddf_grid(work, 256), 256, 0, s>>>(n, p->opts.coarsen_rows, p->nblocks, p->nchunks,
                                                               p->blk_chunk, p->chunk_q0, p->chunk_meta, p->seq,
                                                               p->starts, p->esplit, err);
            ddf_count_launch();
        }
        if (cudaGetLastError() != cudaSuccess) {
            res = DDF_ERR_CUDA;
            break;
        }
        int32_t h = ok;
        if (cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            res = DDF_ERR_CUDA;
            break;
        }
        if (h != ok) res = (ddf_status)h;
    } while (false);
    (void)cudaGetLastError();
    ddf_free(err, s);
    ddf_free(pos, s);
    return res;
}

}  // extern "C"
