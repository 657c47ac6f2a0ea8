/*
 * CPU oracle, symbolic part: elimination tree, column structures of L,
 * supernode partition and the per-supernode index sets used by selected
 * inversion.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, obviously correct
 * restatement of the definitions; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark call it.  It shares no code with the GPU
 * library.
 *
 * Definitions followed:
 *  - structural symmetry of A is assumed (Sec. II-A);
 *  - column structure of L: struct(j) = {j} u {i > j : A_ij != 0}
 *      u  U_{children c of j} (struct(c) \ {c});  parent(j) = min(struct(j)\{j})
 *    (the elimination tree that the paper traverses, Sec. I / II-B);
 *  - supernodes: maximal runs of contiguous columns with the same structure
 *    below and a dense diagonal block, optionally capped in size or relaxed
 *    (Sec. II-A);
 *  - C = {I > K : L_{I,K} != 0} of Alg. 1 / Eq. (newset), kept at the
 *    element level as the row list of supernode K below its own columns.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_PATTERN (-2)
#define ORC_ERR_OOM (-5)

typedef struct {
    int32_t n, nsuper;
    int32_t *parent;     /* column elimination tree [n], -1 = root           */
    int64_t *cstruct_ptr;/* [n+1] offsets of the column structures           */
    int32_t *cstruct;    /* struct(j), ascending, first entry j               */
    int32_t *super_ptr;  /* [nsuper+1] first column of each supernode        */
    int32_t *sparent;    /* [nsuper] supernodal parent, -1 = root            */
    int64_t *rowptr;     /* [nsuper+1] offsets into rows                     */
    int32_t *rows;       /* rows of each supernode: its columns, then C      */
    int64_t nnz_true;    /* sum_j |struct(j)|                                */
} orc_sym;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void orc_sym_free(orc_sym *h) {
    if (!h) return;
    free(h->parent); free(h->cstruct_ptr); free(h->cstruct);
    free(h->super_ptr); free(h->sparent); free(h->rowptr); free(h->rows);
    free(h);
}

/*
 * Symbolic analysis of the lower triangle (CSC, rows ascending, row >= col)
 * of a structurally symmetric matrix.
 *   kind 0: fundamental supernodes, at most `cap` columns.  Column j+1 joins
 *           j's supernode iff parent(j) = j+1, j+1 has exactly one child,
 *           |struct(j+1)| = |struct(j)| - 1 and the supernode has < cap columns.
 *   kind 1: fundamental, then relaxed: walking the supernodes in order, the
 *           group ending at supernode K merges into K+1 iff its parent is
 *           K+1, the merged group has <= cap columns and its explicit zeros
 *           are <= fill * (stored lower entries of the merged group).
 * Returns a handle (NULL on error, *err set).
 */
orc_sym *orc_symbolic(int32_t n, const int64_t *colptr, const int32_t *rowind,
                      int kind, int cap, double fill, int *err) {
    *err = ORC_OK;
    if (n < 0 || cap < 1) { *err = ORC_ERR_ARG; return NULL; }
    orc_sym *h = (orc_sym *)calloc(1, sizeof(orc_sym));
    h->n = n;
    h->parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *nchild = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    int32_t *child_head = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *child_next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t j = 0; j < n; j++) { child_head[j] = -1; mark[j] = -1; }
    int64_t cap_struct = colptr[n] + 16;
    int32_t *cs = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap_struct);
    int64_t *csp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    csp[0] = 0;
    for (int32_t j = 0; j < n; j++) {
        int32_t cnt = 0;
        mark[j] = j; work[cnt++] = j;
        for (int64_t k = colptr[j]; k < colptr[j + 1]; k++) {
            int32_t i = rowind[k];
            if (i < j || i >= n) { *err = ORC_ERR_PATTERN; goto fail; }
            if (mark[i] != j) { mark[i] = j; work[cnt++] = i; }
        }
        for (int32_t c = child_head[j]; c >= 0; c = child_next[c]) {
            for (int64_t k = csp[c]; k < csp[c + 1]; k++) {
                int32_t i = cs[k];
                if (i == c) continue;
                if (mark[i] != j) { mark[i] = j; work[cnt++] = i; }
            }
        }
        qsort(work, (size_t)cnt, sizeof(int32_t), cmp_i32);
        if (csp[j] + cnt > cap_struct) {
            while (csp[j] + cnt > cap_struct) cap_struct *= 2;
            int32_t *ncs = (int32_t *)realloc(cs, sizeof(int32_t) * (size_t)cap_struct);
            if (!ncs) { *err = ORC_ERR_OOM; goto fail; }
            cs = ncs;
        }
        memcpy(cs + csp[j], work, sizeof(int32_t) * (size_t)cnt);
        csp[j + 1] = csp[j] + cnt;
        h->parent[j] = cnt > 1 ? work[1] : -1;
        if (cnt > 1) {
            int32_t p = work[1];
            nchild[p]++;
            child_next[j] = child_head[p];
            child_head[p] = j;
        }
    }
    h->cstruct = cs; h->cstruct_ptr = csp;
    h->nnz_true = csp[n];

    /* fundamental supernodes */
    int32_t *fptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t nf = 0;
    for (int32_t j = 0; j < n; j++) {
        int join = 0;
        if (j > 0) {
            int32_t prev = j - 1;
            int32_t size = j - fptr[nf - 1];
            if (h->parent[prev] == j && nchild[j] == 1 &&
                (csp[j + 1] - csp[j]) == (csp[prev + 1] - csp[prev]) - 1 && size < cap)
                join = 1;
        }
        if (!join) fptr[nf++] = j;
    }
    fptr[nf] = n;

    /* group fundamental supernodes (relaxed merge when kind == 1) */
    int32_t *gptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nf + 1));
    int32_t ng = 0;
    int32_t *col2f = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t f = 0; f < nf; f++)
        for (int32_t j = fptr[f]; j < fptr[f + 1]; j++) col2f[j] = f;
    if (nf > 0) {
        int32_t gstart = 0;                   /* first fundamental supernode of the group */
        int64_t gtrue = 0;                    /* true nonzeros of the group's columns     */
        for (int32_t j = fptr[0]; j < fptr[1]; j++) gtrue += csp[j + 1] - csp[j];
        for (int32_t f = 1; f <= nf; f++) {
            int merge = 0;
            int64_t ftrue = 0;
            if (f < nf) {
                for (int32_t j = fptr[f]; j < fptr[f + 1]; j++) ftrue += csp[j + 1] - csp[j];
                if (kind == 1) {
                    int32_t last = f - 1;     /* last member of the group */
                    int32_t lastcol = fptr[last + 1] - 1;
                    int32_t par = h->parent[lastcol];
                    int32_t gpar = par >= 0 ? col2f[par] : -1;
                    int64_t s = (int64_t)(fptr[f + 1] - fptr[gstart]);
                    int64_t sf = fptr[f + 1] - fptr[f];
                    int64_t cf = (csp[fptr[f] + 1] - csp[fptr[f]]) - sf;
                    int64_t stored = s * (s + 1) / 2 + s * cf;
                    int64_t zeros = stored - (gtrue + ftrue);
                    if (gpar == f && s <= cap && (double)zeros <= fill * (double)stored) merge = 1;
                }
            }
            if (merge) {
                gtrue += ftrue;
            } else {
                gptr[ng++] = fptr[gstart];
                gstart = f;
                gtrue = ftrue;
            }
        }
    }
    gptr[ng] = n;
    h->nsuper = ng;
    h->super_ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ng + 1));
    memcpy(h->super_ptr, gptr, sizeof(int32_t) * (size_t)(ng + 1));

    /* rows of each supernode: its columns, then struct(last column) below it.
     * For a relaxed group this is the union of its members' structures
     * (the structures of later members contain those of earlier ones below
     * their columns). */
    int32_t *col2s = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t K = 0; K < ng; K++)
        for (int32_t j = gptr[K]; j < gptr[K + 1]; j++) col2s[j] = K;
    h->rowptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ng + 1));
    h->rowptr[0] = 0;
    for (int32_t K = 0; K < ng; K++) {
        int32_t f = gptr[K], l = gptr[K + 1] - 1;
        /* union of struct(j) over members, restricted to rows > l, is struct(l) \ {l}
           for fundamental members; build it by marking to stay at the definition */
        int32_t cnt = 0;
        for (int32_t j = f; j <= l; j++)
            for (int64_t k = csp[j]; k < csp[j + 1]; k++) {
                int32_t i = cs[k];
                if (i > l && mark[i] != -2 - K) { mark[i] = -2 - K; work[cnt++] = i; }
            }
        qsort(work, (size_t)cnt, sizeof(int32_t), cmp_i32);
        h->rowptr[K + 1] = h->rowptr[K] + (l - f + 1) + cnt;
    }
    h->rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h->rowptr[ng] > 0 ? h->rowptr[ng] : 1));
    h->sparent = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ng > 0 ? ng : 1));
    for (int32_t K = 0; K < ng; K++) {
        int32_t f = gptr[K], l = gptr[K + 1] - 1;
        int64_t o = h->rowptr[K];
        for (int32_t j = f; j <= l; j++) h->rows[o++] = j;
        int32_t cnt = 0;
        for (int32_t j = f; j <= l; j++)
            for (int64_t k = csp[j]; k < csp[j + 1]; k++) {
                int32_t i = cs[k];
                if (i > l && mark[i] != -100000000 - K) { mark[i] = -100000000 - K; work[cnt++] = i; }
            }
        qsort(work, (size_t)cnt, sizeof(int32_t), cmp_i32);
        memcpy(h->rows + o, work, sizeof(int32_t) * (size_t)cnt);
        h->sparent[K] = cnt > 0 ? col2s[work[0]] : -1;
    }
    free(fptr); free(gptr); free(col2f); free(col2s);
    free(nchild); free(child_head); free(child_next); free(mark); free(work);
    return h;
fail:
    h->cstruct = cs; h->cstruct_ptr = csp;
    free(nchild); free(child_head); free(child_next); free(mark); free(work);
    orc_sym_free(h);
    return NULL;
}

/* field ids for orc_sym_get */
enum { F_PARENT = 0, F_CSTRUCT_PTR, F_CSTRUCT, F_SUPER_PTR, F_SPARENT, F_ROWPTR, F_ROWS, F_NSUPER, F_NNZ_TRUE };

/* Copies field `field` into dst (if not NULL); returns its element count. */
int64_t orc_sym_get(const orc_sym *h, int field, void *dst) {
    int64_t cnt = 0; size_t esz = 4; const void *src = NULL;
    switch (field) {
    case F_PARENT: cnt = h->n; src = h->parent; break;
    case F_CSTRUCT_PTR: cnt = h->n + 1; src = h->cstruct_ptr; esz = 8; break;
    case F_CSTRUCT: cnt = h->cstruct_ptr[h->n]; src = h->cstruct; break;
    case F_SUPER_PTR: cnt = h->nsuper + 1; src = h->super_ptr; break;
    case F_SPARENT: cnt = h->nsuper; src = h->sparent; break;
    case F_ROWPTR: cnt = h->nsuper + 1; src = h->rowptr; esz = 8; break;
    case F_ROWS: cnt = h->rowptr[h->nsuper]; src = h->rows; break;
    case F_NSUPER: return h->nsuper;
    case F_NNZ_TRUE: return h->nnz_true;
    default: return -1;
    }
    if (dst && cnt > 0) memcpy(dst, src, esz * (size_t)cnt);
    return cnt;
}

/*
 * Index sets of the traversal, written out from the definitions, for
 * comparison with the library's plan:
 *   level[K]  = depth of K in the supernodal elimination tree (root 0);
 *   for each K, C (rows of K below its columns) split into maximal runs that
 *   belong to one ancestor supernode J ("segments"): seg_owner = J,
 *   seg_start = first position in C, seg_coloff = C[start] - first column of J;
 *   relidx: for segment t and every position p >= seg_start in C, the
 *   position of C[p] in the row list of J (Alg. 1's "find the collection of
 *   indices" made explicit at the element level).
 * Arrays are allocated by the caller from the sizes returned by a first call
 * with NULL outputs (nseg_total, nrel_total).
 */
int orc_plan(int32_t nsuper, const int32_t *super_ptr, const int32_t *sparent,
             const int64_t *rowptr, const int32_t *rows,
             int32_t *level, int64_t *seg_ptr, int32_t *seg_owner, int32_t *seg_start,
             int32_t *seg_coloff, int64_t *rel_ptr, int32_t *relidx,
             int64_t *nseg_total, int64_t *nrel_total) {
    int32_t n = super_ptr[nsuper];
    int32_t *col2s = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t K = 0; K < nsuper; K++)
        for (int32_t j = super_ptr[K]; j < super_ptr[K + 1]; j++) col2s[j] = K;
    int64_t nseg = 0, nrel = 0;
    for (int32_t K = nsuper - 1; K >= 0; K--) {
        if (level) level[K] = sparent[K] < 0 ? 0 : level[sparent[K]] + 1;
    }
    for (int32_t K = 0; K < nsuper; K++) {
        int32_t s = super_ptr[K + 1] - super_ptr[K];
        int64_t c = rowptr[K + 1] - rowptr[K] - s;
        const int32_t *C = rows + rowptr[K] + s;
        if (seg_ptr) seg_ptr[K] = nseg;
        int64_t p = 0;
        while (p < c) {
            int32_t J = col2s[C[p]];
            int64_t q = p;
            while (q < c && col2s[C[q]] == J) q++;
            if (seg_owner) {
                seg_owner[nseg] = J;
                seg_start[nseg] = (int32_t)p;
                seg_coloff[nseg] = C[p] - super_ptr[J];
                rel_ptr[nseg] = nrel;
                const int32_t *RJ = rows + rowptr[J];
                int64_t mJ = rowptr[J + 1] - rowptr[J];
                for (int64_t r = p; r < c; r++) {
                    int64_t pos = -1;
                    for (int64_t t = 0; t < mJ; t++)
                        if (RJ[t] == C[r]) { pos = t; break; }
                    if (pos < 0) { free(col2s); return ORC_ERR_PATTERN; }
                    relidx[nrel + (r - p)] = (int32_t)pos;
                }
            }
            nseg++;
            nrel += c - p;
            p = q;
        }
    }
    if (seg_ptr) { seg_ptr[nsuper] = nseg; if (rel_ptr) rel_ptr[nseg] = nrel; }
    *nseg_total = nseg;
    *nrel_total = nrel;
    free(col2s);
    return ORC_OK;
}
