// Host symbolic analysis (prerequisite of the plan): elimination tree, column
// structures of L, supernode partition (Sec. II-A), supernodal tree.
//
// Algorithms: the elimination tree by Liu's ancestor-path-compression
// method; the structure of L by row subtrees (row i of L is the union of
// the tree paths from each k with A_ik != 0 up to i), which emits every
// column's rows in ascending order without sorting.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "selinv.h"

struct selinv_analysis_s {
    int32_t n = 0;
    int32_t nsuper = 0;
    int64_t nnz_true = 0;
    std::vector<int32_t> parent, super_ptr, sparent, rows;
    std::vector<int64_t> cptr, rowptr;
    std::vector<int32_t> cind;  // struct(j) without the diagonal, ascending
};

static int analyse_impl(int32_t n, const int64_t *colptr, const int32_t *rowind, int kind,
                        int32_t cap, double fill, selinv_analysis_s *a) {
    a->n = n;
    // ---- strictly lower entries by row: for each row i, columns k < i ----
    std::vector<int64_t> rptr(n + 1, 0);
    for (int32_t j = 0; j < n; j++) {
        int32_t prev = -1;
        for (int64_t e = colptr[j]; e < colptr[j + 1]; e++) {
            int32_t i = rowind[e];
            if (i < j || i >= n || i <= prev) return SELINV_ERR_BAD_PATTERN;
            prev = i;
            if (i > j) rptr[i + 1]++;
        }
    }
    for (int32_t i = 0; i < n; i++) rptr[i + 1] += rptr[i];
    std::vector<int32_t> rcol(rptr[n] > 0 ? rptr[n] : 1);
    {
        std::vector<int64_t> fillp(rptr.begin(), rptr.end() - 1);
        for (int32_t j = 0; j < n; j++)
            for (int64_t e = colptr[j]; e < colptr[j + 1]; e++)
                if (rowind[e] > j) rcol[fillp[rowind[e]]++] = j;
    }
    // ---- elimination tree (Liu) ----
    a->parent.assign(n, -1);
    std::vector<int32_t> anc(n, -1);
    for (int32_t i = 0; i < n; i++) {
        for (int64_t e = rptr[i]; e < rptr[i + 1]; e++) {
            int32_t r = rcol[e];
            while (anc[r] != -1 && anc[r] != i) {
                int32_t nx = anc[r];
                anc[r] = i;
                r = nx;
            }
            if (anc[r] == -1) {
                anc[r] = i;
                a->parent[r] = i;
            }
        }
    }
    // ---- column structures by row subtrees (two passes: count, fill) ----
    std::vector<int32_t> mark(n, -1);
    std::vector<int64_t> ccount(n, 0);
    for (int32_t i = 0; i < n; i++) {
        mark[i] = i;
        for (int64_t e = rptr[i]; e < rptr[i + 1]; e++)
            for (int32_t j = rcol[e]; mark[j] != i; j = a->parent[j]) {
                ccount[j]++;
                mark[j] = i;
            }
    }
    a->cptr.assign(n + 1, 0);
    for (int32_t j = 0; j < n; j++) a->cptr[j + 1] = a->cptr[j] + ccount[j];
    a->cind.resize(a->cptr[n] > 0 ? a->cptr[n] : 1);
    {
        std::vector<int64_t> fillp(a->cptr.begin(), a->cptr.end() - 1);
        std::fill(mark.begin(), mark.end(), -1);
        for (int32_t i = 0; i < n; i++) {
            mark[i] = i;
            for (int64_t e = rptr[i]; e < rptr[i + 1]; e++)
                for (int32_t j = rcol[e]; mark[j] != i; j = a->parent[j]) {
                    a->cind[fillp[j]++] = i;
                    mark[j] = i;
                }
        }
    }
    a->nnz_true = a->cptr[n] + n;
    // ---- fundamental supernodes ----
    std::vector<int32_t> nchild(n, 0);
    for (int32_t j = 0; j < n; j++)
        if (a->parent[j] >= 0) nchild[a->parent[j]]++;
    auto cnt = [&](int32_t j) { return a->cptr[j + 1] - a->cptr[j] + 1; };  // |struct(j)|
    std::vector<int32_t> fstart;
    fstart.reserve(n + 1);
    for (int32_t j = 0; j < n; j++) {
        bool join = false;
        if (j > 0) {
            int32_t size = j - fstart.back();
            join = a->parent[j - 1] == j && nchild[j] == 1 && cnt(j) == cnt(j - 1) - 1 && size < cap;
        }
        if (!join) fstart.push_back(j);
    }
    int32_t nf = (int32_t)fstart.size();
    fstart.push_back(n);
    std::vector<int32_t> col2f(n);
    for (int32_t f = 0; f < nf; f++)
        for (int32_t j = fstart[f]; j < fstart[f + 1]; j++) col2f[j] = f;
    // ---- relaxed merging of a group into the next fundamental supernode ----
    std::vector<int32_t> gstart;
    gstart.reserve(nf + 1);
    if (nf > 0) {
        int32_t g0 = 0;
        int64_t gtrue = 0;
        for (int32_t j = fstart[0]; j < fstart[1]; j++) gtrue += cnt(j);
        for (int32_t f = 1; f <= nf; f++) {
            bool merge = false;
            int64_t ftrue = 0;
            if (f < nf) {
                for (int32_t j = fstart[f]; j < fstart[f + 1]; j++) ftrue += cnt(j);
                if (kind == 1) {
                    int32_t lastcol = fstart[f] - 1;
                    int32_t par = a->parent[lastcol];
                    int64_t s = fstart[f + 1] - fstart[g0];
                    int64_t cf = cnt(fstart[f]) - (fstart[f + 1] - fstart[f]);
                    int64_t stored = s * (s + 1) / 2 + s * cf;
                    int64_t zeros = stored - (gtrue + ftrue);
                    merge = par >= 0 && col2f[par] == f && s <= cap &&
                            (double)zeros <= fill * (double)stored;
                }
            }
            if (merge) {
                gtrue += ftrue;
            } else {
                gstart.push_back(fstart[g0]);
                g0 = f;
                gtrue = ftrue;
            }
        }
    }
    a->nsuper = (int32_t)gstart.size();
    gstart.push_back(n);
    a->super_ptr = gstart;
    // ---- supernode rows: own columns, then struct(last column) below it ----
    const int32_t ns = a->nsuper;
    std::vector<int32_t> col2s(n);
    for (int32_t K = 0; K < ns; K++)
        for (int32_t j = gstart[K]; j < gstart[K + 1]; j++) col2s[j] = K;
    a->rowptr.assign(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) {
        int32_t l = gstart[K + 1] - 1;
        a->rowptr[K + 1] = a->rowptr[K] + (gstart[K + 1] - gstart[K]) + (a->cptr[l + 1] - a->cptr[l]);
    }
    a->rows.resize(a->rowptr[ns] > 0 ? a->rowptr[ns] : 1);
    a->sparent.assign(ns, -1);
    for (int32_t K = 0; K < ns; K++) {
        int32_t f = gstart[K], l = gstart[K + 1] - 1;
        int64_t o = a->rowptr[K];
        for (int32_t j = f; j <= l; j++) a->rows[o++] = j;
        for (int64_t e = a->cptr[l]; e < a->cptr[l + 1]; e++) a->rows[o++] = a->cind[e];
        if (a->cptr[l + 1] > a->cptr[l]) a->sparent[K] = col2s[a->cind[a->cptr[l]]];
    }
    return SELINV_OK;
}

extern "C" int selinv_analyse(int32_t n, const int64_t *colptr, const int32_t *rowind, int kind,
                              int32_t cap, double fill, selinv_analysis *out) {
    if (!out || n < 0 || cap < 1 || (n > 0 && (!colptr || !rowind)) || (kind != 0 && kind != 1) ||
        !(fill >= 0.0))
        return SELINV_ERR_INVALID_ARG;
    *out = nullptr;
    selinv_analysis_s *a = new (std::nothrow) selinv_analysis_s();
    if (!a) return SELINV_ERR_OOM;
    int rc;
    try {
        rc = analyse_impl(n, colptr, rowind, kind, cap, fill, a);
    } catch (const std::bad_alloc &) {
        rc = SELINV_ERR_OOM;
    }
    if (rc != SELINV_OK) {
        delete a;
        return rc;
    }
    *out = a;
    return SELINV_OK;
}

extern "C" int64_t selinv_analysis_get(selinv_analysis a, int field, void *dst) {
    if (!a) return SELINV_ERR_INVALID_ARG;
    const void *src = nullptr;
    int64_t cnt = 0;
    size_t esz = 4;
    switch (field) {
    case 0: src = a->parent.data(); cnt = a->n; break;
    case 3: src = a->super_ptr.data(); cnt = a->nsuper + 1; break;
    case 4: src = a->sparent.data(); cnt = a->nsuper; break;
    case 5: src = a->rowptr.data(); cnt = a->nsuper + 1; esz = 8; break;
    case 6: src = a->rows.data(); cnt = a->rowptr[a->nsuper]; break;
    case 7: return a->nsuper;
    case 8: return a->nnz_true;
    default: return SELINV_ERR_INVALID_ARG;
    }
    if (dst && cnt > 0) std::memcpy(dst, src, esz * (size_t)cnt);
    return cnt;
}

extern "C" void selinv_analysis_destroy(selinv_analysis a) { delete a; }
