// Plan serialisation: ddf_plan_save writes a plan (descriptors, work units,
// level order, the plan's copies of indices and values) into a host buffer;
// ddf_plan_load rebuilds a device plan from it without re-inspection.  This is
// the amortisation the paper argues for (Sec. V-C): the inspector runs once
// per pattern and its result is reused.
//
// Layout: a fixed header (magic, version, sizes, options) followed by the
// arrays in a fixed order, each 8-byte aligned, and an FNV-1a checksum of
// everything before it.  The buffer is host-endian; load it on a machine of
// the same byte order.
#include <string.h>

#include <vector>

#include "ddf_internal.cuh"

namespace {

constexpr char MAGIC[8] = {'D', 'D', 'F', 'P', 'L', 'A', 'N', '1'};
constexpr int32_t VERSION = 6;

struct Header {
    char magic[8];
    int32_t version, kind, n, n_cols, depth, has_values, vdtype, mrhs_units_per_ticket;
    int32_t nlevels, nblocks, mrhs_nmat;
    int64_t nnz, npts, ncod, ncod_type[3], nunits[3], nchunks;
    int64_t ntiles[2];
    ddf_opts opts;
};

struct Piece {
    void* dev;     // device array (save: source; load: destination)
    size_t bytes;
};

size_t pad8(size_t b) { return (b + 7) & ~(size_t)7; }

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 14695981039346656037ull;  // 64-bit FNV offset basis
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

size_t value_size(int32_t dt) { return dt == DDF_F32 ? 4 : (dt == DDF_BF16 ? 2 : 8); }

// The arrays of a plan in file order (pointers of p; sizes from the header).
// slots[k] receives the address of the plan field that holds piece k.
std::vector<Piece> pieces(ddf_plan_s* p, const Header& h, void** slots[24]) {
    const int64_t n = h.n, nv = h.kind == DDF_SPMV ? h.nnz : h.npts;
    const bool tr = h.kind == DDF_SPTRSV;
    const bool lp = h.vdtype != DDF_F64;
    std::vector<Piece> v;
    int k = 0;
    auto add = [&](void** ptr, size_t bytes) {
        slots[k++] = ptr;
        v.push_back(Piece{*ptr, bytes});
    };
    add((void**)&p->starts, 4 * (size_t)(n + 1));
    add((void**)&p->col, 4 * (size_t)nv);
    add((void**)&p->val, 8 * (size_t)nv);
    add((void**)&p->part_ptr, 4 * (size_t)(h.depth + 1));
    add((void**)&p->cod, sizeof(dcod) * (size_t)h.ncod);
    for (int t = 0; t < 3; ++t) add((void**)&p->units[t], sizeof(dunit) * (size_t)h.nunits[t]);
    if (!tr)
        for (int t = 0; t < 2; ++t) add((void**)&p->tiles[t], sizeof(dtile) * (size_t)h.ntiles[t]);
    if (tr) {
        add((void**)&p->seq, 4 * (size_t)n);
        add((void**)&p->dinv, 8 * (size_t)n);
        add((void**)&p->orig_rowptr, 4 * (size_t)(n + 1));
        if (h.opts.lower_of_input) add((void**)&p->orig_rowend, 4 * (size_t)n);
        if (h.nblocks > 0) {
            add((void**)&p->blk_ptr, 4 * (size_t)(h.nblocks + 1));
            add((void**)&p->esplit, 4 * (size_t)n);
            add((void**)&p->qcod, 4 * (size_t)n);
            add((void**)&p->chunk_q0, 4 * (size_t)(h.nchunks + 1));
            add((void**)&p->chunk_meta, 4 * (size_t)h.nchunks);
            add((void**)&p->blk_chunk, 4 * (size_t)(h.nblocks + 1));
        }
        // a batch plan: its matrices' first rows, from which the load rebuilds the multi-RHS solve's items
        if (h.mrhs_nmat > 0) add((void**)&p->mrhs_moff, 4 * (size_t)h.mrhs_nmat);
    }
    if (lp) {
        add((void**)&p->val_lp, value_size(h.vdtype) * (size_t)nv);
        if (tr) {
            add((void**)&p->dinv_lp, 4 * (size_t)n);
            add((void**)&p->diag, 8 * (size_t)n);
        }
    }
    return v;
}

Header header_of(ddf_plan_s* p) {
    Header h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, MAGIC, 8);
    h.version = VERSION;
    h.kind = p->kind;
    h.n = p->n;
    h.n_cols = p->n_cols;
    h.depth = p->depth;
    h.has_values = p->has_values;
    h.vdtype = p->vdtype;
    h.mrhs_units_per_ticket = p->mrhs_units_per_ticket;
    h.nlevels = p->nlevels;
    h.nblocks = p->nblocks;
    h.mrhs_nmat = p->mrhs_nmat;
    h.nchunks = p->nchunks;
    h.nnz = p->nnz;
    h.npts = p->npts;
    h.ncod = p->ncod;
    for (int t = 0; t < 3; ++t) {
        h.ncod_type[t] = p->ncod_type[t];
        h.nunits[t] = p->nunits[t];
    }
    for (int t = 0; t < 2; ++t) h.ntiles[t] = p->ntiles[t];
    h.opts = p->opts;
    return h;
}

size_t total_bytes(const std::vector<Piece>& v) {
    size_t b = pad8(sizeof(Header));
    for (const Piece& x : v) b += pad8(x.bytes);
    return b + sizeof(uint64_t);
}

}  // namespace

extern "C" {

ddf_status ddf_plan_save(ddf_plan_t p, void* buf, size_t* len) {
    ddf_nvtx_range nvtx_("ddf_plan_save");
    if (!p || !len) return DDF_ERR_ARG;
    Header h = header_of(p);
    void** slots[24];
    std::vector<Piece> v = pieces(p, h, slots);
    const size_t need = total_bytes(v);
    if (!buf) {
        *len = need;
        return DDF_OK;
    }
    if (*len < need) {
        *len = need;
        return DDF_ERR_ARG;
    }
    unsigned char* out = (unsigned char*)buf;
    memset(out, 0, need);
    memcpy(out, &h, sizeof(h));
    size_t off = pad8(sizeof(Header));
    cudaStream_t s = p->stream;
    for (const Piece& x : v) {
        if (x.bytes > 0) DDF_CUDA_TRY(cudaMemcpyAsync(out + off, x.dev, x.bytes, cudaMemcpyDeviceToHost, s));
        off += pad8(x.bytes);
    }
    DDF_CUDA_TRY(cudaStreamSynchronize(s));
    const uint64_t sum = fnv1a(out, off);
    memcpy(out + off, &sum, sizeof(sum));
    *len = need;
    return DDF_OK;
}

ddf_status ddf_plan_load(const void* buf, size_t len, ddf_stream_t stream, ddf_plan_t* out) {
    ddf_nvtx_range nvtx_("ddf_plan_load");
    if (!out) return DDF_ERR_ARG;
    *out = nullptr;
    if (!buf || len < pad8(sizeof(Header)) + sizeof(uint64_t)) return DDF_ERR_ARG;
    Header h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, MAGIC, 8) != 0 || h.version != VERSION) return DDF_ERR_ARG;
    if ((h.kind != DDF_SPMV && h.kind != DDF_SPTRSV) || h.n < 0 || h.n_cols < 0 || h.depth < 0 || h.nnz < 0 ||
        h.npts < 0 || h.ncod < 0 || h.nunits[0] < 0 || h.nunits[1] < 0 || h.nunits[2] < 0 ||
        (h.vdtype != DDF_F64 && h.vdtype != DDF_F32 && h.vdtype != DDF_BF16))
        return DDF_ERR_ARG;
    // every counted element takes at least one byte of the buffer: this bounds
    // the sizes below (no overflow) before they are summed
    const int64_t cap = (int64_t)len;
    if (h.nblocks < 0 || h.nlevels < 0 || h.nchunks < 0 || h.nchunks > (int64_t)len || (h.nblocks > 0 && (h.kind != DDF_SPTRSV || h.opts.coarsen_rows < 1)))
        return DDF_ERR_ARG;
    if (h.mrhs_nmat < 0 || (h.mrhs_nmat > 0 && (h.kind != DDF_SPTRSV || h.mrhs_nmat > h.n || h.nblocks > 0)))
        return DDF_ERR_ARG;
    if (h.n >= cap || h.depth >= cap || h.nblocks >= cap || h.nnz > cap || h.npts > cap || h.ncod > cap || h.nunits[0] > cap ||
        h.nunits[1] > cap || h.nunits[2] > cap || h.ntiles[0] < 0 || h.ntiles[1] < 0 || h.ntiles[0] > cap ||
        h.ntiles[1] > cap || (h.kind == DDF_SPTRSV && h.ntiles[0] + h.ntiles[1] != 0))
        return DDF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ddf_plan_s* p = nullptr;
    ddf_status st = ddf_new_plan((ddf_kind)h.kind, &h.opts, s, h.n, h.n_cols, h.nnz, &p);
    if (st) return st;
    p->depth = h.depth;
    p->npts = h.npts;
    p->ncod = h.ncod;
    p->has_values = h.has_values;
    p->vdtype = h.vdtype;
    p->mrhs_units_per_ticket = h.mrhs_units_per_ticket;
    p->nlevels = h.nlevels;
    p->nblocks = h.nblocks;
    p->nchunks = h.nchunks;
    for (int t = 0; t < 3; ++t) {
        if (h.ncod_type[t] < 0) st = DDF_ERR_ARG;
        p->ncod_type[t] = h.ncod_type[t];
        p->nunits[t] = h.nunits[t];
    }
    for (int t = 0; t < 2; ++t) p->ntiles[t] = h.ntiles[t];
    if (st) {
        ddf_plan_destroy(p);
        return st;
    }
    void** slots[24];
    std::vector<Piece> v = pieces(p, h, slots);
    const unsigned char* in = (const unsigned char*)buf;
    const size_t need = total_bytes(v);
    if (len < need) {
        ddf_plan_destroy(p);
        return DDF_ERR_ARG;
    }
    size_t off = pad8(sizeof(Header));
    for (const Piece& x : v) off += pad8(x.bytes);
    uint64_t sum = 0;
    memcpy(&sum, in + off, sizeof(sum));
    if (sum != fnv1a(in, off)) {
        ddf_plan_destroy(p);
        return DDF_ERR_ARG;
    }
    off = pad8(sizeof(Header));
    for (size_t i = 0; i < v.size() && !st; ++i) {
        const size_t b = v[i].bytes;
        if (b > 0) {
            void* d = nullptr;
            // 16 spare bytes: val / col / val_lp are staged by 16-byte-granular bulk copies
            if (ddf_alloc_injected_failure() || cudaMallocAsync(&d, b + 16, s) != cudaSuccess) {
                (void)cudaGetLastError();
                st = DDF_ERR_OOM;
                break;
            }
            *slots[i] = d;
            if (cudaMemcpyAsync(d, in + off, b, cudaMemcpyHostToDevice, s) != cudaSuccess) st = DDF_ERR_CUDA;
        }
        off += pad8(b);
    }
    // refinement scratch of a low-precision SpTRSV plan
    if (!st && h.vdtype != DDF_F64 && h.kind == DDF_SPTRSV && h.n > 0) {
        st = ddf_alloc(&p->r64, h.n, s);
        if (!st) st = ddf_alloc(&p->rlp, h.n, s);
        if (!st) st = ddf_alloc(&p->xlp, h.n, s);
        if (!st) st = ddf_alloc(&p->nrm, 3, s);
    }
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (!st) st = ddf_plan_validate(p);
    // derived from the validated units: the solve's unit positions, the
    // SpMV's long PSC II rows
    if (!st && h.kind == DDF_SPTRSV) st = ddf_build_unit_q(p, s);
    // a batch plan's multi-RHS solve items, rebuilt from the matrices' first
    // rows once those are checked (0 first, non-decreasing, within n)
    if (!st && h.mrhs_nmat > 0) {
        std::vector<int32_t> moff((size_t)h.mrhs_nmat);
        int32_t* dmoff = p->mrhs_moff;
        p->mrhs_moff = nullptr;
        p->mrhs_nmat = 0;
        if (cudaMemcpyAsync(moff.data(), dmoff, 4 * moff.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = DDF_ERR_CUDA;
        ddf_free(dmoff, s);
        for (size_t i = 0; !st && i < moff.size(); ++i)
            if ((i == 0 && moff[0] != 0) || (i > 0 && moff[i] < moff[i - 1]) || moff[i] > h.n) st = DDF_ERR_ARG;
        if (!st) st = ddf_build_mrhs_items(p, moff.data(), h.mrhs_nmat, s);
    }
    if (!st && h.kind == DDF_SPMV) st = ddf_build_long_rows(p, s);
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (st) {
        (void)cudaGetLastError();
        ddf_plan_destroy(p);
        return st;
    }
    *out = p;
    return DDF_OK;
}

}  // extern "C"
