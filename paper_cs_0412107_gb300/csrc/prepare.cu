// prepare.cu -- host-side preparation of a matrix for the sweep (Sec. 2):
// CSR validation (D must be non-singular, Sec. 2.2), the rows of C^dagger
// that Eq. 5 runs over, the Gauss-Seidel dependency levels of C and C^dagger,
// and the chunk stream the sweep stages into shared memory.  Shared by the
// single-matrix handle and the pool.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "prepare.h"

namespace mcinv {

static mcinv_status prep_fail(std::string *err, mcinv_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (err) *err = buf;
    return st;
}

mcinv_status prepare_matrix(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                            int min_blob, Prepared &P, std::string *err)
{
    const int NV = cplx ? 2 : 1;
    if (n <= 0 || n > (1LL << 30)) return prep_fail(err, MCINV_E_ARG, "n = %lld out of range", (long long)n);
    if (!row_ptr || !col || !val) return prep_fail(err, MCINV_E_ARG, "NULL CSR array");
    if (row_ptr[0] != 0) return prep_fail(err, MCINV_E_ARG, "row_ptr[0] != 0");
    const int64_t nnz = row_ptr[n];
    if (nnz < n || nnz > (1LL << 31) - 1) return prep_fail(err, MCINV_E_ARG, "nnz = %lld out of range", (long long)nnz);
    P.n = n;
    P.nnz = nnz;
    P.cplx = cplx;
    // ---- host validation: sorted unique columns in range, diagonal present and usable
    std::vector<double> diag((size_t)n * NV);
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return prep_fail(err, MCINV_E_ARG, "row_ptr decreases at row %lld", (long long)i);
        bool has_diag = false;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int64_t j = col[e];
            if (j < 0 || j >= n) return prep_fail(err, MCINV_E_ARG, "column %lld out of range in row %lld", (long long)j, (long long)i);
            if (e > row_ptr[i] && col[e - 1] >= j) return prep_fail(err, MCINV_E_ARG, "columns not strictly increasing in row %lld", (long long)i);
            for (int v = 0; v < NV; ++v)
                if (!std::isfinite(val[e * NV + v])) return prep_fail(err, MCINV_E_ARG, "non-finite value in row %lld", (long long)i);
            if (j == i) {
                has_diag = true;
                for (int v = 0; v < NV; ++v) diag[(size_t)i * NV + v] = val[e * NV + v];
            }
        }
        bool zero = true;
        for (int v = 0; v < NV; ++v) zero &= diag[(size_t)i * NV + v] == 0.0;
        if (!has_diag || zero)
            return prep_fail(err, MCINV_E_SINGULAR_DIAG, "diagonal entry of row %lld is %s", (long long)i, has_diag ? "zero" : "missing");
    }

    // ---- C^dagger rows: (C^H)_{j,i} = conj(c_ij), off-diagonal only, columns ascending
    std::vector<int64_t> wcount(n + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] != i) wcount[col[e] + 1]++;
    for (int64_t j = 0; j < n; ++j) wcount[j + 1] += wcount[j];
    std::vector<int32_t> wcol(wcount[n]);
    std::vector<double> wval((size_t)wcount[n] * NV);
    {
        std::vector<int64_t> fill(wcount.begin(), wcount.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const int64_t j = col[e];
                if (j == i) continue;
                const int64_t p = fill[j]++;
                wcol[p] = (int32_t)i;
                wval[p * NV] = val[e * NV];
                if (cplx) wval[p * NV + 1] = -val[e * NV + 1];
            }
    }

    // ---- dependency levels: row i waits for every j < i it reads this cycle
    //      through C (Eq. 4) or C^dagger (Eq. 5)
    std::vector<int32_t> level(n, 0);
    int nlev = 0;
    for (int64_t i = 0; i < n; ++i) {
        int lv = 0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1] && col[e] < i; ++e) lv = std::max(lv, level[col[e]] + 1);
        for (int64_t e = wcount[i]; e < wcount[i + 1] && wcol[e] < i; ++e) lv = std::max(lv, level[wcol[e]] + 1);
        level[i] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    P.nlev = nlev;
    // pieces of a row: 1 up to SPLIT_ENTRIES entries on either side, 2 up to twice that, else 4
    auto pieces_of = [&](int64_t i) {
        const int64_t dz = row_ptr[i + 1] - row_ptr[i] - 1, dw = wcount[i + 1] - wcount[i];
        const int64_t dm = std::max(dz, dw);
        return dm <= SPLIT_ENTRIES ? 1 : dm <= 2 * SPLIT_ENTRIES ? 2 : 4;
    };
    std::vector<int32_t> lev_ptr(nlev + 1, 0), perm(n);
    for (int64_t i = 0; i < n; ++i) lev_ptr[level[i] + 1]++;
    for (int l = 0; l < nlev; ++l) lev_ptr[l + 1] += lev_ptr[l];
    {
        std::vector<int32_t> fill(lev_ptr.begin(), lev_ptr.end() - 1);
        for (int64_t i = 0; i < n; ++i) perm[fill[level[i]]++] = (int32_t)i;
        // rows of one level are independent: order them by decreasing number of
        // pieces (so every split row's items start at a multiple of its P), then
        // by decreasing work, so the rows a warp takes together cost about the same
        for (int l = 0; l < nlev; ++l)
            std::stable_sort(perm.begin() + lev_ptr[l], perm.begin() + lev_ptr[l + 1], [&](int32_t x, int32_t y) {
                const int px = pieces_of(x), py = pieces_of(y);
                if (px != py) return px > py;
                const int64_t dx = (row_ptr[x + 1] - row_ptr[x]) + (wcount[x + 1] - wcount[x]);
                const int64_t dy = (row_ptr[y + 1] - row_ptr[y]) + (wcount[y + 1] - wcount[y]);
                return dx > dy;
            });
    }

    // ---- the chunk stream (see internal.h): per chunk of a level, the row
    //      records, constants (filled on the GPU below) and entries of C and C^H
    const size_t ent_sz = cplx ? sizeof(EntC) : sizeof(EntR);
    const size_t cst_sz = cplx ? sizeof(CstC) : sizeof(CstR);
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    auto blob_bytes = [&](size_t rows, size_t items, size_t nz, size_t nwv) {
        return a16(16 * (items + 1)) + a16(cst_sz * rows) + a16(ent_sz * nz) + a16(ent_sz * nwv);
    };
    auto zdeg = [&](int64_t i) { return (size_t)(row_ptr[i + 1] - row_ptr[i] - 1); };
    auto wdeg = [&](int64_t i) { return (size_t)(wcount[i + 1] - wcount[i]); };
    size_t blob_max = (size_t)min_blob;
    for (int64_t i = 0; i < n; ++i) blob_max = std::max(blob_max, blob_bytes(1, pieces_of(i), zdeg(i), wdeg(i)));
    blob_max = (blob_max + 127) & ~(size_t)127;
    if (blob_max > 100 * 1024)
        return prep_fail(err, MCINV_E_UNSUPPORTED,
                         "a row has too many off-diagonal entries in C and C^dagger for one shared-memory chunk (limit about %zu)",
                         (size_t)(100 * 1024 - 64) / ent_sz);
    P.blob_max = (int)blob_max;
    std::vector<ChunkDesc> chunks;
    std::vector<long long> cst_at(n);
    size_t stream_bytes = 0;
    for (int l = 0; l < nlev; ++l) {
        int64_t p = lev_ptr[l];
        while (p < lev_ptr[l + 1]) {
            const int64_t pb = p;
            size_t nz = 0, nwv = 0, items = 0;
            while (p < lev_ptr[l + 1] &&
                   blob_bytes(p - pb + 1, items + pieces_of(perm[p]), nz + zdeg(perm[p]), nwv + wdeg(perm[p])) <= blob_max) {
                nz += zdeg(perm[p]);
                nwv += wdeg(perm[p]);
                items += pieces_of(perm[p]);
                ++p;
            }
            ChunkDesc d{};
            d.rows = (int)(p - pb);
            d.items = (int)items;
            d.pb = (int)pb;
            d.cst_off = (int)a16(16 * (items + 1));
            d.zent_off = d.cst_off + (int)a16(cst_sz * d.rows);
            d.went_off = d.zent_off + (int)a16(ent_sz * nz);
            d.bytes = d.went_off + (int)a16(ent_sz * nwv);
            d.off = (long long)stream_bytes;
            d.flags = (p == lev_ptr[l + 1] ? CHUNK_LEVEL_END : 0) | (items > (size_t)d.rows ? CHUNK_SPLIT : 0);
            stream_bytes += ((size_t)d.bytes + 127) & ~(size_t)127;
            chunks.push_back(d);
        }
    }
    std::vector<uint8_t> stream(stream_bytes, 0);
    for (const ChunkDesc &d : chunks) {
        uint8_t *blob = stream.data() + d.off;
        RowMeta *meta = (RowMeta *)blob;
        int zo = 0, wo = 0, it = 0;
        for (int r = 0; r < d.rows; ++r) {
            const int64_t i = perm[d.pb + r];
            cst_at[d.pb + r] = d.off + d.cst_off + (long long)(r * cst_sz);
            const int np = pieces_of(i);
            const int lg = np == 1 ? 0 : np == 2 ? 1 : 2;
            const int dz = (int)zdeg(i), dw = (int)wdeg(i);
            const int cz = (dz + np - 1) / np, cw = (dw + np - 1) / np;  // entries per piece
            for (int k = 0; k < np; ++k)
                meta[it + k] = RowMeta{(int)i, zo + std::min(dz, k * cz), wo + std::min(dw, k * cw), k | (lg << 2) | (r << 4)};
            it += np;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                if (col[e] == i) continue;
                if (!cplx) ((EntR *)(blob + d.zent_off))[zo++] = EntR{col[e], (float)val[e]};
                else ((EntC *)(blob + d.zent_off))[zo++] = EntC{col[e], (float)val[2 * e], (float)val[2 * e + 1], 0};
            }
            for (int64_t e = wcount[i]; e < wcount[i + 1]; ++e) {
                if (!cplx) ((EntR *)(blob + d.went_off))[wo++] = EntR{wcol[e], (float)wval[e]};
                else ((EntC *)(blob + d.went_off))[wo++] = EntC{wcol[e], (float)wval[2 * e], (float)wval[2 * e + 1], 0};
            }
        }
        meta[d.items] = RowMeta{-1, zo, wo, 0};
    }
    // ---- the flat form (GridRow records) for the grid-wide sweep
    {
        std::vector<GridRow> grow(n + 1);
        size_t tz = 0, tw = 0;
        for (int64_t p = 0; p < n; ++p) {
            tz += zdeg(perm[p]);
            tw += wdeg(perm[p]);
        }
        std::vector<uint8_t> gz(std::max<size_t>(tz, 1) * ent_sz, 0), gw(std::max<size_t>(tw, 1) * ent_sz, 0);
        int zb = 0, wb = 0;
        for (int64_t p = 0; p < n; ++p) {
            const int64_t i = perm[p];
            const int np = pieces_of(i);
            const int lg = np == 1 ? 0 : np == 2 ? 1 : 2;
            const int dz = (int)zdeg(i), dw = (int)wdeg(i);
            if (dz > GRID_DEG_MAX || dw > GRID_DEG_MAX)
                return prep_fail(err, MCINV_E_UNSUPPORTED, "row %lld has more than %d off-diagonal entries", (long long)i, GRID_DEG_MAX);
            grow[p] = GridRow{(int)i, zb, wb, lg | (dz << 2) | (dw << 17)};
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                if (col[e] == i) continue;
                if (!cplx) ((EntR *)gz.data())[zb++] = EntR{col[e], (float)val[e]};
                else ((EntC *)gz.data())[zb++] = EntC{col[e], (float)val[2 * e], (float)val[2 * e + 1], 0};
            }
            for (int64_t e = wcount[i]; e < wcount[i + 1]; ++e) {
                if (!cplx) ((EntR *)gw.data())[wb++] = EntR{wcol[e], (float)wval[e]};
                else ((EntC *)gw.data())[wb++] = EntC{wcol[e], (float)wval[2 * e], (float)wval[2 * e + 1], 0};
            }
        }
        grow[n] = GridRow{-1, zb, wb, 0};
        P.grow = std::move(grow);
        P.gzent = std::move(gz);
        P.gwent = std::move(gw);
        P.lev_ptr = lev_ptr;
    }
    std::vector<int32_t> pos(n);
    for (int64_t p = 0; p < n; ++p) pos[perm[p]] = (int32_t)p;
    std::vector<double> diag_pos((size_t)n * NV);
    for (int64_t p = 0; p < n; ++p)
        for (int v = 0; v < NV; ++v) diag_pos[(size_t)p * NV + v] = diag[(size_t)perm[p] * NV + v];

    P.chunks = std::move(chunks);
    P.stream = std::move(stream);
    P.cst_at = std::move(cst_at);
    P.perm = std::move(perm);
    P.pos = std::move(pos);
    P.diag_pos = std::move(diag_pos);
    return MCINV_OK;
}

mcinv_status color_order(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                         std::vector<int32_t> &order, int *ncolors, std::string *err)
{
    const int NV = cplx ? 2 : 1;
    if (n <= 0 || n > (1LL << 30)) return prep_fail(err, MCINV_E_ARG, "n = %lld out of range", (long long)n);
    if (!row_ptr || !col) return prep_fail(err, MCINV_E_ARG, "NULL CSR array");
    if (row_ptr[0] != 0) return prep_fail(err, MCINV_E_ARG, "row_ptr[0] != 0");
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return prep_fail(err, MCINV_E_ARG, "row_ptr decreases at row %lld", (long long)i);
        bool has_diag = false, zero = true;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int64_t j = col[e];
            if (j < 0 || j >= n) return prep_fail(err, MCINV_E_ARG, "column %lld out of range in row %lld", (long long)j, (long long)i);
            if (e > row_ptr[i] && col[e - 1] >= j) return prep_fail(err, MCINV_E_ARG, "columns not strictly increasing in row %lld", (long long)i);
            if (j == i) {
                has_diag = true;
                if (val)
                    for (int v = 0; v < NV; ++v) zero &= val[e * NV + v] == 0.0;
                else
                    zero = false;
            }
        }
        if (!has_diag || zero)
            return prep_fail(err, MCINV_E_SINGULAR_DIAG, "diagonal entry of row %lld is %s", (long long)i, has_diag ? "zero" : "missing");
    }
    // lower neighbours of every row in C + C^T: j < i with c_ij != 0 (row i) or c_ji != 0 (column i)
    std::vector<int64_t> tptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] > i) tptr[col[e] + 1]++;
    for (int64_t j = 0; j < n; ++j) tptr[j + 1] += tptr[j];
    std::vector<int32_t> trow(tptr[n]);
    {
        std::vector<int64_t> fill(tptr.begin(), tptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                if (col[e] > i) trow[fill[col[e]]++] = (int32_t)i;  // row i < col[e] reads col[e]'s column
    }
    std::vector<int32_t> color(n, 0);
    std::vector<int64_t> mark;  // mark[c] == i: colour c is taken by a neighbour of row i
    int nc = 0;
    for (int64_t i = 0; i < n; ++i) {
        auto take = [&](int64_t j) {
            const int c = color[j];
            if ((size_t)c >= mark.size()) mark.resize(c + 1, -1);
            mark[c] = i;
        };
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1] && col[e] < i; ++e) take(col[e]);
        for (int64_t e = tptr[i]; e < tptr[i + 1]; ++e) take(trow[e]);
        int c = 0;
        while ((size_t)c < mark.size() && mark[c] == i) ++c;
        color[i] = c;
        nc = std::max(nc, c + 1);
    }
    std::vector<int64_t> cptr(nc + 1, 0);
    for (int64_t i = 0; i < n; ++i) cptr[color[i] + 1]++;
    for (int c = 0; c < nc; ++c) cptr[c + 1] += cptr[c];
    order.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) order[cptr[color[i]]++] = (int32_t)i;
    if (ncolors) *ncolors = nc;
    return MCINV_OK;
}

void permute_csr(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                 const std::vector<int32_t> &order, std::vector<int64_t> &rp2, std::vector<int32_t> &col2,
                 std::vector<double> &val2)
{
    const int NV = cplx ? 2 : 1;
    std::vector<int32_t> inv(n);
    for (int64_t k = 0; k < n; ++k) inv[order[k]] = (int32_t)k;
    rp2.assign(n + 1, 0);
    for (int64_t k = 0; k < n; ++k) rp2[k + 1] = rp2[k] + (row_ptr[order[k] + 1] - row_ptr[order[k]]);
    col2.resize(rp2[n]);
    val2.resize((size_t)rp2[n] * NV);
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t i = order[k];
        row.clear();
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) row.emplace_back(inv[col[e]], e);
        std::sort(row.begin(), row.end());
        int64_t o = rp2[k];
        for (const auto &pr : row) {
            col2[o] = pr.first;
            for (int v = 0; v < NV; ++v) val2[(size_t)o * NV + v] = val[(size_t)pr.second * NV + v];
            ++o;
        }
    }
}

}  // namespace mcinv

extern "C" mcinv_status mcinv_color_order(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t *order,
                                          int32_t *ncolors)
{
    if (!order) return MCINV_E_ARG;
    std::vector<int32_t> ord;
    int nc = 0;
    const mcinv_status st = mcinv::color_order(n, row_ptr, col, nullptr, 0, ord, &nc, nullptr);
    if (st != MCINV_OK) return st;
    std::copy(ord.begin(), ord.end(), order);
    if (ncolors) *ncolors = nc;
    return MCINV_OK;
}
