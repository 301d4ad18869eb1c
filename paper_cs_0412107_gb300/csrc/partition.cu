// partition.cu -- the block partition of Sec. 4, on the host.
//
// The paper suggests cutting C into small non-singular diagonal blocks D_b
// (around zeros or small values of the diagonal) and sweeping block by block.
// With S = blockdiag(S_b), S_b the principal square root of D_b (S_b = 1 for a
// block of one row), the block sweep
//   z_b <- S_b^-1 phi_b - D_b^-1 sum_{c != b} C_bc z_c
//   w_b <- S_b^-H phi_b - D_b^-H sum_{c != b} (C^H)_bc w_c
// is exactly the row sweep of Eqs. 4/5 on C~ = S^-1 C S^-1 (whose diagonal
// blocks are the identity, so rows of one block never read each other), with
// z = S^-1 z~ and w = S^-H w~: E[z w^H] = S^-1 C~^-1 S^-1 = C^-1.  So the device
// runs the ordinary sweep on C~; this file builds C~ and S_b^-1.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <vector>

#include "partition.h"

namespace mcinv {

using cd = std::complex<double>;

static mcinv_status part_fail(std::string *err, mcinv_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (err) *err = buf;
    return st;
}

// In-place inverse of a b x b matrix (row-major) by Gauss-Jordan elimination with
// partial pivoting; false if a pivot vanishes.
static bool invert(int b, std::vector<cd> &a)
{
    std::vector<cd> inv(b * b, 0.0);
    for (int i = 0; i < b; ++i) inv[i * b + i] = 1.0;
    for (int c = 0; c < b; ++c) {
        int p = c;
        for (int r = c + 1; r < b; ++r)
            if (std::abs(a[r * b + c]) > std::abs(a[p * b + c])) p = r;
        if (!(std::abs(a[p * b + c]) > 0.0)) return false;
        if (p != c)
            for (int k = 0; k < b; ++k) {
                std::swap(a[p * b + k], a[c * b + k]);
                std::swap(inv[p * b + k], inv[c * b + k]);
            }
        const cd d = 1.0 / a[c * b + c];
        for (int k = 0; k < b; ++k) {
            a[c * b + k] *= d;
            inv[c * b + k] *= d;
        }
        for (int r = 0; r < b; ++r) {
            if (r == c) continue;
            const cd f = a[r * b + c];
            if (f == 0.0) continue;
            for (int k = 0; k < b; ++k) {
                a[r * b + k] -= f * a[c * b + k];
                inv[r * b + k] -= f * inv[c * b + k];
            }
        }
    }
    a = inv;
    return true;
}

// The principal square root S of D and S^-1 by the Denman-Beavers iteration
// (Denman & Beavers 1976): Y0 = D, Z0 = I, Y <- (Y + Z^-1)/2, Z <- (Z + Y^-1)/2,
// with Y -> D^(1/2) and Z -> D^(-1/2) when D has no eigenvalue on the closed
// negative real axis.  Returns false when it does not converge.
static bool sqrt_pair(int b, const std::vector<cd> &D, std::vector<cd> &Y, std::vector<cd> &Z)
{
    Y = D;
    Z.assign(b * b, 0.0);
    for (int i = 0; i < b; ++i) Z[i * b + i] = 1.0;
    double scale = 0.0;
    for (const cd &x : D) scale = std::max(scale, std::abs(x));
    for (int it = 0; it < 100; ++it) {
        std::vector<cd> Yi = Y, Zi = Z;
        if (!invert(b, Yi) || !invert(b, Zi)) return false;
        double change = 0.0, size = 0.0;
        for (int k = 0; k < b * b; ++k) {
            const cd y = 0.5 * (Y[k] + Zi[k]);
            const cd z = 0.5 * (Z[k] + Yi[k]);
            change = std::max(change, std::abs(y - Y[k]));
            size = std::max(size, std::abs(y));
            Y[k] = y;
            Z[k] = z;
        }
        if (!std::isfinite(change)) return false;
        if (change <= 1e-15 * size) {
            // check: Z D Z = I
            double res = 0.0;
            for (int i = 0; i < b; ++i)
                for (int j = 0; j < b; ++j) {
                    cd s = 0.0;
                    for (int k = 0; k < b; ++k)
                        for (int l = 0; l < b; ++l) s += Z[i * b + k] * D[k * b + l] * Z[l * b + j];
                    res = std::max(res, std::abs(s - (i == j ? 1.0 : 0.0)));
                }
            return res < 1e-10 && scale > 0.0;
        }
    }
    return false;
}

mcinv_status partition_transform(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                                 int64_t nblocks, const int64_t *block_ptr, std::vector<int64_t> &rp2,
                                 std::vector<int32_t> &col2, std::vector<double> &val2, Partition &part,
                                 std::string *err)
{
    const int NV = cplx ? 2 : 1;
    if (nblocks < 1 || nblocks > n || !block_ptr) return part_fail(err, MCINV_E_ARG, "bad block partition");
    if (block_ptr[0] != 0 || block_ptr[nblocks] != n)
        return part_fail(err, MCINV_E_ARG, "block_ptr must start at 0 and end at n");
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t sz = block_ptr[b + 1] - block_ptr[b];
        if (sz < 1 || sz > MCINV_MAX_PARTITION_BLOCK)
            return part_fail(err, MCINV_E_ARG, "block %lld has %lld rows (1..%d allowed)", (long long)b, (long long)sz,
                             MCINV_MAX_PARTITION_BLOCK);
    }
    if (!row_ptr || !col || !val || row_ptr[0] != 0) return part_fail(err, MCINV_E_ARG, "bad CSR arrays");
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return part_fail(err, MCINV_E_ARG, "row_ptr decreases at row %lld", (long long)i);
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] < 0 || col[e] >= n) return part_fail(err, MCINV_E_ARG, "column out of range in row %lld", (long long)i);
    }
    std::vector<int32_t> blk(n);
    for (int64_t b = 0; b < nblocks; ++b)
        for (int64_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i) blk[i] = (int32_t)b;
    auto value = [&](int64_t e) { return cplx ? cd(val[2 * e], val[2 * e + 1]) : cd(val[e], 0.0); };

    // S_b^-1 of every block of two or more rows (one-row blocks keep S = 1)
    part.block_ptr.assign(block_ptr, block_ptr + nblocks + 1);
    part.sinv_off.assign(nblocks + 1, 0);
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t sz = block_ptr[b + 1] - block_ptr[b];
        part.sinv_off[b + 1] = part.sinv_off[b] + (sz > 1 ? sz * sz : 0);
    }
    part.sinv.assign(part.sinv_off[nblocks], 0.0);
    part.s.assign(part.sinv_off[nblocks], 0.0);
    part.multi = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        const int b0 = (int)block_ptr[b], sz = (int)(block_ptr[b + 1] - block_ptr[b]);
        if (sz == 1) continue;
        ++part.multi;
        std::vector<cd> D(sz * sz, 0.0), Y, Z;
        for (int r = 0; r < sz; ++r)
            for (int64_t e = row_ptr[b0 + r]; e < row_ptr[b0 + r + 1]; ++e)
                if (col[e] >= b0 && col[e] < b0 + sz) D[r * sz + (col[e] - b0)] = value(e);
        if (!sqrt_pair(sz, D, Y, Z))
            return part_fail(err, MCINV_E_SINGULAR_DIAG,
                             "diagonal block %lld (rows %d..%d) has no principal square root (it is singular or "
                             "has an eigenvalue on the closed negative real axis)",
                             (long long)b, b0, b0 + sz - 1);
        if (!cplx)
            for (std::vector<cd> *m : {&Y, &Z})
                for (cd &z : *m) {
                    if (std::abs(z.imag()) > 1e-12 * (1.0 + std::abs(z.real())))
                        return part_fail(err, MCINV_E_SINGULAR_DIAG, "diagonal block %lld has no real principal square root", (long long)b);
                    z = cd(z.real(), 0.0);
                }
        std::copy(Z.begin(), Z.end(), part.sinv.begin() + part.sinv_off[b]);
        std::copy(Y.begin(), Y.end(), part.s.begin() + part.sinv_off[b]);
    }
    auto sinv = [&](int64_t b, int r, int c) -> cd {  // (S_b^-1)_{rc}
        const int64_t sz = block_ptr[b + 1] - block_ptr[b];
        if (sz == 1) return 1.0;
        return part.sinv[part.sinv_off[b] + r * sz + c];
    };
    // one-row blocks need a usable diagonal of their own
    for (int64_t b = 0; b < nblocks; ++b) {
        if (block_ptr[b + 1] - block_ptr[b] != 1) continue;
        const int64_t i = block_ptr[b];
        bool ok = false;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col[e] == i && std::abs(value(e)) > 0.0) ok = true;
        if (!ok) return part_fail(err, MCINV_E_SINGULAR_DIAG, "diagonal entry of row %lld is zero or missing", (long long)i);
    }

    // C~ = S^-1 C S^-1, block row by block row: C~_bc = S_b^-1 C_bc S_c^-1 for c != b;
    // C~_bb = I for a block of two or more rows, c_ii for one row
    rp2.assign(n + 1, 0);
    col2.clear();
    val2.clear();
    for (int64_t b = 0; b < nblocks; ++b) {
        const int b0 = (int)block_ptr[b], sb = (int)(block_ptr[b + 1] - block_ptr[b]);
        // T = S_b^-1 C[rows of b, :] as sparse rows (column -> value)
        std::vector<std::map<int32_t, cd>> T(sb);
        for (int r = 0; r < sb; ++r)
            for (int k = 0; k < sb; ++k) {
                const cd f = sinv(b, r, k);
                if (f == 0.0) continue;
                for (int64_t e = row_ptr[b0 + k]; e < row_ptr[b0 + k + 1]; ++e) T[r][col[e]] += f * value(e);
            }
        for (int r = 0; r < sb; ++r) {
            std::map<int32_t, cd> out;
            for (const auto &kv : T[r]) {
                const int32_t j = kv.first;
                const int64_t c = blk[j];
                if (c == b) continue;
                const int c0 = (int)block_ptr[c], sc = (int)(block_ptr[c + 1] - block_ptr[c]);
                for (int t = 0; t < sc; ++t) {  // column j of C_bc times row (j - c0) of S_c^-1
                    const cd f = sinv(c, j - c0, t);
                    if (f != 0.0) out[c0 + t] += kv.second * f;
                }
            }
            if (sb == 1) {
                cd d = 0.0;
                for (int64_t e = row_ptr[b0]; e < row_ptr[b0 + 1]; ++e)
                    if (col[e] == b0) d = value(e);
                out[b0] = d;
            } else {
                out[b0 + r] = 1.0;
            }
            for (const auto &kv : out) {
                if (kv.second == 0.0) continue;
                col2.push_back(kv.first);
                val2.push_back(kv.second.real());
                if (cplx) val2.push_back(kv.second.imag());
            }
            rp2[b0 + r + 1] = (int64_t)col2.size();
        }
    }
    (void)NV;
    if (col2.size() > (size_t)((1LL << 31) - 1)) return part_fail(err, MCINV_E_ARG, "C~ has too many nonzeros");
    return MCINV_OK;
}

}  // namespace mcinv
