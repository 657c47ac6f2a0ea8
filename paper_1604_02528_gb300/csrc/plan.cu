// Plan construction (selinv_symbolic), schedules and the C ABI of the
// numeric phase.  The plan makes Alg. 1's "find the collection of indices C"
// explicit once: every C is split into runs owned by one ancestor supernode,
// and the row of each C entry inside its owner's row list (relative index)
// is stored, so that the kernels gather A^{-1}_{C,C} without searching.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "nvtx.h"
#include "plan.h"

namespace selinv {

static std::atomic<int64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

size_t elem_size(int dtype) { return dtype == SELINV_F64 ? 8 : 16; }

template <typename X, typename A>
static int upload(X **dptr, const std::vector<X, A> &h) {
    *dptr = nullptr;
    size_t bytes = sizeof(X) * (h.empty() ? 1 : h.size());
    if (cudaMalloc((void **)dptr, bytes) != cudaSuccess) return SELINV_ERR_OOM;
    if (!h.empty() && cudaMemcpy(*dptr, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SELINV_ERR_CUDA;
    return SELINV_OK;
}

static void dfree(void *p) {
    if (p) cudaFree(p);
}

void Workspace::release() {
    if (!owned.empty()) {
        // the buffers' own device: its kernels must be done with them, and
        // the reuse cache files them under that device
        DeviceGuard g(device);
        cudaDeviceSynchronize();   // no kernel may still use a buffer that goes into the cache
        for (auto &o : owned) dev_release(o.first, o.second);
        owned.clear();
    }
    LDu = Vt = nullptr;
    ticket = nullptr;
    partial_all = nullptr;
    colexpZ = tcount = nullptr;
    yacc = nullptr;
    lhs = nullptr;
    lhsu = nullptr;
    colexp = colexpY = nullptr;
    dacc = nullptr;
    linvd = nullptr;
    linvexp = nullptr;
    LD = Linv = partial = nullptr;
    counter = done = nullptr;
    work = nullptr;
    bytes_elem = 0;
}

// a workspace buffer of `bytes`, recorded for release
template <typename X> static bool wget(Workspace &w, X **ptr, size_t bytes) {
    void *v = nullptr;
    if (dev_alloc(&v, bytes) != cudaSuccess) return false;
    w.owned.emplace_back(v, bytes);
    *ptr = static_cast<X *>(v);
    return true;
}

int Workspace::ensure(const PlanData &p, int dtype) {
    const size_t es = elem_size(dtype);
    if (LD && bytes_elem >= es) return SELINV_OK;
    release();
    DeviceGuard g(p.device);
    device = p.device;
    if (!wget(*this, &LD, es * (size_t)std::max<int64_t>(p.nnz, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &Linv, es * (size_t)std::max<int64_t>(p.linv_total, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &partial, es * (size_t)std::max<int64_t>(p.part_max, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &counter, sizeof(int) * (size_t)std::max(p.ns, 1))) return SELINV_ERR_OOM;
    // one extra flag (index ns) that nothing ever sets: the target of the timeout test
    if (!wget(*this, &done, sizeof(int) * (size_t)(p.ns + 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &ticket, sizeof(int))) return SELINV_ERR_OOM;
    if (!wget(*this, &work, es * (size_t)std::max<int64_t>(p.nnz, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &lhs, sizeof(uint16_t) * (size_t)std::max<int64_t>(p.lhs_total, 8)))
        return SELINV_ERR_OOM;
    // tcgen05 operand layout of the Lhat digits: real, or the complex operand
    const int64_t nlhsu = std::max<int64_t>(dtype == SELINV_F64 ? p.lhsu_total : std::max(p.lhsu_total, p.lhsuz_total), 8);
    if (!wget(*this, &lhsu, sizeof(uint16_t) * (size_t)nlhsu)) return SELINV_ERR_OOM;
    cudaMemset(lhsu, 0, sizeof(uint16_t) * (size_t)nlhsu);   // padding stays zero
    if (!wget(*this, &colexp, sizeof(int) * (size_t)std::max(p.n, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &colexpY, sizeof(int) * (size_t)std::max(p.n, 1))) return SELINV_ERR_OOM;
    const size_t dwords = (dtype == SELINV_F64 ? 2 : 4) * (size_t)std::max<int64_t>(p.linv_total, 1);
    if (!wget(*this, &dacc, sizeof(long long) * dwords)) return SELINV_ERR_OOM;
    if (!wget(*this, &colexpZ, sizeof(int) * (size_t)std::max(p.n, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &linvexp, sizeof(int) * (size_t)std::max(p.n, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &linvd, sizeof(uint16_t) * (size_t)std::max<int64_t>(p.linvd_total, 8)))
        return SELINV_ERR_OOM;
    cudaMemset(linvd, 0, sizeof(uint16_t) * (size_t)std::max<int64_t>(p.linvd_total, 8));   // padding rows stay zero
    cudaMemset(colexpZ, 0, sizeof(int) * (size_t)std::max(p.n, 1));
    const size_t ny = (dtype == SELINV_F64 && p.lhs_total > 0) ? 2 * (size_t)p.nnz : 2;
    if (!wget(*this, &yacc, sizeof(long long) * ny)) return SELINV_ERR_OOM;
    if (!wget(*this, &tcount, sizeof(int) * (size_t)std::max<int64_t>(p.tile_total, 1)))
        return SELINV_ERR_OOM;
    cudaMemset(yacc, 0, sizeof(long long) * ny);
    cudaMemset(tcount, 0, sizeof(int) * (size_t)std::max<int64_t>(p.tile_total, 1));
    cudaMemset(colexpY, 0, sizeof(int) * (size_t)std::max(p.n, 1));
    cudaMemset(dacc, 0, sizeof(long long) * dwords);
    cudaMemset(counter, 0, sizeof(int) * (size_t)std::max(p.ns, 1));
    cudaMemset(done, 0, sizeof(int) * (size_t)(p.ns + 1));
    cudaMemset(ticket, 0, sizeof(int));
    // the zeroing above runs on the legacy default stream, which a caller's
    // non-blocking stream does not wait for: finish it before any kernel can
    // see the buffers (reused ones hold a previous plan's data)
    if (cudaDeviceSynchronize() != cudaSuccess) return SELINV_ERR_CUDA;
    bytes_elem = es;
    return SELINV_OK;
}

// the LU form's extra scratch (element size of the current workspace)
int Workspace::ensure_lu(const PlanData &p) {
    if (LDu) return SELINV_OK;
    DeviceGuard g(device);
    if (!wget(*this, &LDu, bytes_elem * (size_t)std::max<int64_t>(p.nnz, 1))) return SELINV_ERR_OOM;
    if (!wget(*this, &Vt, bytes_elem * (size_t)std::max<int64_t>(p.linv_total, 1))) return SELINV_ERR_OOM;
    return SELINV_OK;
}

int Workspace::ensure_persistent(const PlanData &p) {
    if (partial_all) return SELINV_OK;
    DeviceGuard g(device);
    if (!wget(*this, &partial_all, bytes_elem * (size_t)std::max<int64_t>(p.part_all, 1)))
        return SELINV_ERR_OOM;
    return SELINV_OK;
}

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------
static int build_plan(PlanData &p, int32_t n, int32_t ns, const int32_t *super_ptr,
                      const int32_t *sparent, const int64_t *rowptr, const int32_t *rowind) {
    p.n = n;
    p.ns = ns;
    if (super_ptr[0] != 0 || super_ptr[ns] != n) return SELINV_ERR_INVALID_ARG;
    for (int32_t K = 0; K < ns; K++)
        if (super_ptr[K + 1] <= super_ptr[K]) return SELINV_ERR_INVALID_ARG;
    if (rowptr[0] != 0) return SELINV_ERR_INVALID_ARG;
    p.super_ptr.assign(super_ptr, super_ptr + ns + 1);
    p.sparent.assign(sparent, sparent + ns);
    p.rowptr.assign(rowptr, rowptr + ns + 1);
    const int64_t nrows = rowptr[ns];
    p.rows.assign(rowind, rowind + nrows);
    std::vector<int32_t> col2s(n);
    for (int32_t K = 0; K < ns; K++)
        for (int32_t j = super_ptr[K]; j < super_ptr[K + 1]; j++) col2s[j] = K;
    // structure checks
    p.panel_off.assign(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) {
        const int32_t fc = super_ptr[K], s = super_ptr[K + 1] - fc;
        const int64_t m = rowptr[K + 1] - rowptr[K];
        if (m < s) return SELINV_ERR_BAD_PATTERN;
        if (s > SELINV_MAX_SUPERNODE) return SELINV_ERR_UNSUPPORTED;  // widest column tile of the kernels
        const int32_t *R = rowind + rowptr[K];
        for (int32_t j = 0; j < s; j++)
            if (R[j] != fc + j) return SELINV_ERR_BAD_PATTERN;
        for (int64_t r = 1; r < m; r++)
            if (R[r] <= R[r - 1] || R[r] >= n) return SELINV_ERR_BAD_PATTERN;
        const int32_t par = sparent[K];
        if (m > s) {
            if (par != col2s[R[s]]) return SELINV_ERR_BAD_ETREE;
        } else if (par != -1) {
            return SELINV_ERR_BAD_ETREE;
        }
        p.panel_off[K + 1] = p.panel_off[K] + m * s;
    }
    p.nnz = p.panel_off[ns];
    // levels (depth from the root); parents have larger indices
    p.level.assign(ns, 0);
    p.nlevels = ns > 0 ? 1 : 0;
    for (int32_t K = ns - 1; K >= 0; K--) {
        p.level[K] = sparent[K] < 0 ? 0 : p.level[sparent[K]] + 1;
        p.nlevels = std::max(p.nlevels, p.level[K] + 1);
    }
    p.level_ptr.assign(p.nlevels + 1, 0);
    for (int32_t K = 0; K < ns; K++) p.level_ptr[p.level[K] + 1]++;
    for (int l = 0; l < p.nlevels; l++) p.level_ptr[l + 1] += p.level_ptr[l];
    p.level_list.assign(ns, 0);
    {
        std::vector<int64_t> f(p.level_ptr.begin(), p.level_ptr.end() - 1);
        for (int32_t K = 0; K < ns; K++) p.level_list[f[p.level[K]]++] = K;
    }
    // owner segments of every C, relative indices (merge walk in the owner's
    // rows).  Pass 1 counts each supernode's segments and relative indices
    // (serial, O(sum c)); pass 2 fills them with the supernodes spread over
    // host threads, each supernode into its own ranges, so that the plan does
    // not depend on the threads.
    std::vector<int64_t> nseg(ns + 1, 0), nrel(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) {
        const int32_t s = super_ptr[K + 1] - super_ptr[K];
        const int64_t c = rowptr[K + 1] - rowptr[K] - s;
        const int32_t *C = rowind + rowptr[K] + s;
        int64_t q = 0, segs = 0, rels = 0;
        while (q < c) {
            const int32_t J = col2s[C[q]];
            if (J <= K) return SELINV_ERR_BAD_PATTERN;
            int64_t qe = q;
            while (qe < c && col2s[C[qe]] == J) qe++;
            segs++;
            rels += c - q;
            q = qe;
        }
        nseg[K + 1] = nseg[K] + segs;
        nrel[K + 1] = nrel[K] + rels;
    }
    const int64_t tseg = nseg[ns], trel = nrel[ns];
    p.seg_ptr.assign(nseg.begin(), nseg.end());
    p.seg_owner.assign(tseg, 0);
    p.seg_start.assign(tseg, 0);
    p.seg_coloff.assign(tseg, 0);
    p.rel_ptr.assign(tseg + 1, 0);
    p.rel_ptr[tseg] = trel;
    // written in full by the fill below (colbase / relbase: C positions there,
    // the diagonal-block positions zeroed there)
    p.relidx.resize(trel);
    p.colbase.resize(nrows > 0 ? nrows : 1);
    p.relbase.resize(nrows > 0 ? nrows : 1);
    if (nrows == 0) p.colbase[0] = p.relbase[0] = 0;
    std::atomic<int> bad{0};
    std::atomic<int32_t> next{0};
    constexpr int32_t kBlock = 16;   // supernodes per claim
    // blocks are claimed from the root end: the supernodes near the root
    // carry the longest row lists, so they start first
    auto fill = [&]() {
        for (;;) {
            const int32_t K1 = ns - next.fetch_add(kBlock);
            if (K1 <= 0 || bad.load(std::memory_order_relaxed)) return;
            for (int32_t K = std::max(0, K1 - kBlock); K < K1; K++) {
                const int32_t s = super_ptr[K + 1] - super_ptr[K];
                const int64_t c = rowptr[K + 1] - rowptr[K] - s;
                const int32_t *C = rowind + rowptr[K] + s;
                int64_t g = nseg[K], rb = nrel[K], q = 0;
                for (int64_t r = 0; r < s; r++) p.colbase[rowptr[K] + r] = p.relbase[rowptr[K] + r] = 0;
                while (q < c) {
                    const int32_t J = col2s[C[q]];
                    int64_t qe = q;
                    while (qe < c && col2s[C[qe]] == J) qe++;
                    const int32_t fcJ = super_ptr[J];
                    const int64_t mJ = rowptr[J + 1] - rowptr[J];
                    const int32_t *RJ = rowind + rowptr[J];
                    p.seg_owner[g] = J;
                    p.seg_start[g] = (int32_t)q;
                    p.seg_coloff[g] = C[q] - fcJ;
                    p.rel_ptr[g] = rb;
                    int64_t t = C[q] - fcJ;  // C[q] is a column of J, at that position of rows(J)
                    for (int64_t r = q; r < c; r++) {
                        while (t < mJ && RJ[t] < C[r]) t++;
                        if (t >= mJ || RJ[t] != C[r]) {   // not closed
                            bad.store(1);
                            return;
                        }
                        p.relidx[rb + (r - q)] = (int32_t)t;
                    }
                    for (int64_t r = q; r < qe; r++) {
                        const int64_t pos = rowptr[K] + s + r;
                        p.colbase[pos] = p.panel_off[J] + (int64_t)(C[r] - fcJ) * mJ;
                        p.relbase[pos] = rb - q;
                    }
                    rb += c - q;
                    g++;
                    q = qe;
                }
            }
        }
    };
    {
        const int64_t work = trel + nrows;
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nthr = work < (1 << 18) ? 1 : (int)std::min<unsigned>(hw, 16u);
        std::vector<std::thread> pool;
        for (int i = 1; i < nthr; i++) pool.emplace_back(fill);
        fill();
        for (auto &th : pool) th.join();
    }
    if (bad.load()) return SELINV_ERR_BAD_PATTERN;
    // L_KK^{-1} offsets; split-partial offsets inside each level
    p.linv_off.assign(ns + 1, 0);
    p.part_off.assign(ns > 0 ? ns : 1, 0);
    p.ntiles.assign(ns > 0 ? ns : 1, 1);
    for (int32_t K = 0; K < ns; K++) {
        const int64_t s = super_ptr[K + 1] - super_ptr[K];
        p.linv_off[K + 1] = p.linv_off[K] + s * s;
        const int64_t c = rowptr[K + 1] - rowptr[K] - s;
        p.ntiles[K] = (int32_t)std::max<int64_t>(1, (c + kTM - 1) / kTM);
    }
    p.linv_total = p.linv_off[ns];
    // digit planes of Lhat for the tensor-core path: 7 planes of s x roundup(c, 16)
    p.lhs_off.assign(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) {
        const int64_t s = super_ptr[K + 1] - super_ptr[K];
        const int64_t c = rowptr[K + 1] - rowptr[K] - s;
        const int64_t c16 = (c + 15) / 16 * 16;
        p.lhs_off[K + 1] = p.lhs_off[K] + (s >= kOzMinS ? 7 * s * c16 : 0);
    }
    p.lhs_total = p.lhs_off[ns];
    p.lhsu_off.assign(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) {
        const int64_t s = super_ptr[K + 1] - super_ptr[K];
        const int64_t c = rowptr[K + 1] - rowptr[K] - s;
        const int64_t c16 = (c + 15) / 16 * 16, s64 = (s + 63) / 64 * 64;
        p.lhsu_off[K + 1] = p.lhsu_off[K] + (s >= kOzMinS ? 7 * s64 * c16 : 0);
    }
    p.lhsu_total = p.lhsu_off[ns];
    // complex symmetric: the operand of 2s rows over k' = 2q + part (2c long)
    p.lhsuz_off.assign(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) {
        const int64_t s = super_ptr[K + 1] - super_ptr[K];
        const int64_t c = rowptr[K + 1] - rowptr[K] - s;
        const int64_t k16 = (2 * c + 15) / 16 * 16, s64 = (2 * s + 63) / 64 * 64;
        p.lhsuz_off[K + 1] = p.lhsuz_off[K] + (s >= kOzMinS ? 7 * s64 * k16 : 0);
    }
    p.lhsuz_total = p.lhsuz_off[ns];
    p.linvd_off.assign(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) {
        const int64_t s = super_ptr[K + 1] - super_ptr[K];
        // supernodes wider than 64 columns may hold the tcgen05 operand layout
        // (rows padded to 128) for the transposed Lhat product
        const int64_t rows = s > 64 ? (s + 63) / 64 * 64 : s;
        p.linvd_off[K + 1] = p.linvd_off[K] + (s >= kOzMinS ? 7 * rows * ((s + 15) / 16 * 16) : 0);
    }
    p.linvd_total = p.linvd_off[ns];
    p.tile_base.assign(ns + 1, 0);
    for (int32_t K = 0; K < ns; K++) p.tile_base[K + 1] = p.tile_base[K] + p.ntiles[K];
    p.tile_total = p.tile_base[ns];
    p.part_max = 1;
    for (int l = 0; l < p.nlevels; l++) {
        int64_t acc = 0;
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t K = p.level_list[e];
            const int64_t s = super_ptr[K + 1] - super_ptr[K];
            p.part_off[K] = acc;
            acc += (int64_t)p.ntiles[K] * s * s;
        }
        p.part_max = std::max(p.part_max, acc);
    }
    p.part_off_all.assign(ns > 0 ? ns : 1, 0);
    p.part_all = 0;
    for (int32_t K = 0; K < ns; K++) {
        const int64_t s = super_ptr[K + 1] - super_ptr[K];
        p.part_off_all[K] = p.part_all;
        p.part_all += (int64_t)p.ntiles[K] * s * s;
    }
    p.part_all = std::max<int64_t>(p.part_all, 1);
    return SELINV_OK;
}

// Device copies of the plan, made on first use (so that plans can be built
// and inspected on a host without a GPU).
int ensure_device(PlanData &p) {
    if (p.d_status) return SELINV_OK;
    if (cudaGetDevice(&p.device) != cudaSuccess) return SELINV_ERR_CUDA;
    static bool configured = false;
    if (!configured) {
        if (configure_selinv_kernels() != cudaSuccess) return SELINV_ERR_CUDA;
        if (configure_ozaki_kernels() != cudaSuccess) return SELINV_ERR_CUDA;
        if (configure_tc_kernels() != cudaSuccess) return SELINV_ERR_CUDA;
        if (configure_tcw_kernels() != cudaSuccess) return SELINV_ERR_CUDA;
        configured = true;
    }
    int rc;
    if ((rc = upload(&p.d_super_ptr, p.super_ptr))) return rc;
    if ((rc = upload(&p.d_sparent, p.sparent))) return rc;
    if ((rc = upload(&p.d_rowptr, p.rowptr))) return rc;
    if ((rc = upload(&p.d_rows, p.rows))) return rc;
    if ((rc = upload(&p.d_panel_off, p.panel_off))) return rc;
    if ((rc = upload(&p.d_colbase, p.colbase))) return rc;
    if ((rc = upload(&p.d_relbase, p.relbase))) return rc;
    if ((rc = upload(&p.d_relidx, p.relidx))) return rc;
    if ((rc = upload(&p.d_linv_off, p.linv_off))) return rc;
    if ((rc = upload(&p.d_part_off, p.part_off))) return rc;
    if ((rc = upload(&p.d_part_off_all, p.part_off_all))) return rc;
    if ((rc = upload(&p.d_lhs_off, p.lhs_off))) return rc;
    if ((rc = upload(&p.d_lhsu_off, p.lhsu_off))) return rc;
    if ((rc = upload(&p.d_lhsuz_off, p.lhsuz_off))) return rc;
    if ((rc = upload(&p.d_tile_base, p.tile_base))) return rc;
    if ((rc = upload(&p.d_linvd_off, p.linvd_off))) return rc;
    if ((rc = upload(&p.d_seg_ptr, p.seg_ptr))) return rc;
    if ((rc = upload(&p.d_seg_start, p.seg_start))) return rc;
    int *st = nullptr;
    if (cudaMalloc((void **)&st, sizeof(int)) != cudaSuccess) return SELINV_ERR_OOM;
    if (cudaMemset(st, 0, sizeof(int)) != cudaSuccess) return SELINV_ERR_CUDA;
    p.d_status = st;
    return SELINV_OK;
}

void PlanData::release_device() {
    dfree(d_super_ptr); dfree(d_sparent); dfree(d_rowptr); dfree(d_rows); dfree(d_panel_off);
    dfree(d_colbase); dfree(d_relbase); dfree(d_relidx); dfree(d_linv_off); dfree(d_part_off); dfree(d_part_off_all);
    dfree(d_lhs_off); dfree(d_lhsu_off); dfree(d_lhsuz_off); dfree(d_tile_base); dfree(d_linvd_off); dfree(d_status); dfree(d_sel_pos);
    dfree(d_seg_ptr); dfree(d_seg_start);
    d_lhs_off = d_lhsu_off = d_lhsuz_off = d_tile_base = d_linvd_off = d_sel_pos = d_seg_ptr = nullptr;
    d_seg_start = nullptr;
    d_super_ptr = d_sparent = d_rows = d_relidx = nullptr;
    d_rowptr = d_panel_off = d_colbase = d_relbase = d_linv_off = d_part_off = d_part_off_all = nullptr;
    d_status = nullptr;
}

ProbDesc make_desc(const PlanData &p, Workspace &w, int dtype, const void *L, const void *D, void *Z,
                   bool persistent) {
    ProbDesc d;
    std::memset(&d, 0, sizeof(d));
    d.super_ptr = p.d_super_ptr;
    d.rowptr = p.d_rowptr;
    d.rows = p.d_rows;
    d.panel_off = p.d_panel_off;
    d.colbase = p.d_colbase;
    d.relbase = p.d_relbase;
    d.relidx = p.d_relidx;
    d.linv_off = p.d_linv_off;
    d.part_off = persistent ? p.d_part_off_all : p.d_part_off;
    d.sparent = p.d_sparent;
    d.seg_ptr = p.d_seg_ptr;
    d.seg_start = p.d_seg_start;
    d.L = L;
    d.D = D;
    d.Z = Z;
    d.Yout = Z;
    d.LD = w.LD;
    d.Linv = w.Linv;
    d.partial = persistent ? w.partial_all : w.partial;
    d.counter = w.counter;
    d.done = persistent ? w.done : nullptr;
    d.status = p.d_status;
    d.lhs = w.lhs;
    d.lhs_off = p.d_lhs_off;
    d.lhsu = w.lhsu;
    d.lhsu_off = dtype == SELINV_F64 ? p.d_lhsu_off : p.d_lhsuz_off;
    d.colexp = w.colexp;
    d.colexpY = w.colexpY;
    d.dacc = w.dacc;
    d.colexpZ = w.colexpZ;
    d.linvd = w.linvd;
    d.linvd_off = p.d_linvd_off;
    d.linvexp = w.linvexp;
    d.yacc = w.yacc;
    d.tcount = w.tcount;
    d.tile_base = p.d_tile_base;
    d.ns = p.ns;
    d.n = p.n;
    d.nnz = p.nnz;
    d.check_gather = (p.opts.debug_checks & 4) ? 1 : 0;
    d.dtype = dtype == SELINV_C128H ? SELINV_C128 : dtype;   // element type of the kernels
    d.herm = dtype == SELINV_C128H;
    d.symmetrize = p.opts.symmetrize;
    return d;
}

// ---------------------------------------------------------------------------
// schedules: the launch sequence of one call (single or batched problems)
// ---------------------------------------------------------------------------
void Schedule::release() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    if (graph_host) cudaGraphExecDestroy(graph_host);
    graph_host = nullptr;
    host_key.fill(nullptr);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_mid) cudaEventDestroy(ev_mid);
    side = nullptr;
    ev_fork = ev_join = ev_mid = nullptr;
    join_at = join_at2 = -1;
    dfree(d_descs); dfree(d_items); dfree(d_work); dfree(d_buckets); dfree(tcslab); dfree(d_red);
    d_descs = nullptr; d_items = nullptr; d_work = nullptr; d_buckets = nullptr; tcslab = nullptr; d_red = nullptr;
}

int build_schedule(Schedule &S, const std::vector<const PlanData *> &plans,
                   const std::vector<ProbDesc> &descs, int mode, bool split_norm) {
    S.release();
    S.launches.clear();
    S.h_items.clear();
    S.h_work.clear();
    S.h_red.clear();
    S.pre_ptr.clear();
    S.pre_bytes.clear();
    S.mode = mode;
    const int np = (int)plans.size();
    // subset selection: supernodes outside every selected entry's ancestor chain do not run
    auto act = [&](int i, int32_t K) { return plans[i]->active.empty() || plans[i]->active[K] != 0; };
    // tensor-core contraction for this problem and width (never for the LU form)
    auto ozok = [&](int i, int s) { return !descs[i].lu && oz_eligible(descs[i].dtype, s, plans[i]->opts); };
    // Lhat of a tensor-core supernode wider than 64 columns: the transposed tcgen05 kernel
    auto lhat_tc = [&](int i, int s) { return plans[i]->opts.fast_contraction == 1 && s > 64; };
    // complex supernodes (symmetric or Hermitian) on tcgen05 (the transposed
    // gather-GEMM and the diagonal block over the real 2c-long contraction;
    // level and plain schedules, not the LU form; their Lhat stays on the FP64 pipe)
    auto zok = [&](int i, int s) {
        const selinv_opts &o = plans[i]->opts;
        return !descs[i].lu && descs[i].dtype == SELINV_C128 && o.fast_contraction == 1 &&
               s >= std::max(kOzMinS, o.oz_min_s) && (mode == SELINV_SCHED_LEVEL || mode == SELINV_SCHED_PLAIN);
    };
    // DFMA supernodes small enough for a warp each (k_selinv_tiny; not the LU form)
    auto tiny = [&](int i, int32_t K) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        return !descs[i].lu && s <= 8 && c <= 64 && !ozok(i, s) && !zok(i, s);
    };
    // Level schedule: the normalization (steps 1, 2, 2b) runs in up to three
    // phases.  The supernodes of the first `ltop` levels -- the top of the
    // tree, a few large supernodes per level whose launches leave most SMs
    // idle -- are normalized first on the main stream; those of the levels
    // [ltop, lmid), then the rest, on a side stream, while the main stream
    // traverses the levels above them (the traversal of a level reads the
    // normalization of its own supernodes only).  The main stream waits for
    // the side stream's first phase before level ltop and for the second
    // before level lmid (two phases: lmid = the number of levels).
    int ltop = 0, lmid = 0;
    int nlev_all = 0;
    for (int i = 0; i < np; i++) nlev_all = std::max(nlev_all, plans[i]->nlevels);
    if (mode == SELINV_SCHED_LEVEL && split_norm) {
        int64_t seen = 0;
        for (int l = 0; l < nlev_all; l++) {
            for (int i = 0; i < np; i++)
                if (l < plans[i]->nlevels) seen += plans[i]->level_ptr[l + 1] - plans[i]->level_ptr[l];
            if (seen <= kTopSupernodes) ltop = l + 1;
            if (seen <= kMidSupernodes) lmid = l + 1;
        }
        if (ltop >= nlev_all) ltop = 0;   // the whole tree is "top": nothing to overlap
        if (ltop == 0 || lmid <= ltop || lmid >= nlev_all) lmid = nlev_all;
    }
    const int nph = ltop == 0 ? 1 : (lmid < nlev_all ? 3 : 2);
    auto phase_of = [&](int i, int32_t K) {
        const int l = plans[i]->level[K];
        return l < ltop ? 0 : (l < lmid ? 1 : 2);
    };
    for (int ph = 0; ph < nph; ph++) {
        const size_t ph_first = S.launches.size();
        // supernodes of this phase (all when there is one phase)
        auto actn = [&](int i, int32_t K) { return act(i, K) && (nph == 1 || phase_of(i, K) == ph); };
        // 1) L_KK^{-1}, Dinv for every supernode (one launch per dtype and size class)
        for (int dt = 0; dt < 2; dt++)
            for (int large = 1; large >= 0; large--) {
                const int64_t off = (int64_t)S.h_work.size();
                for (int i = 0; i < np; i++) {
                    if (descs[i].dtype != dt) continue;
                    const PlanData &p = *plans[i];
                    for (int32_t K = 0; K < p.ns; K++)
                        if (actn(i, K) && (p.super_ptr[K + 1] - p.super_ptr[K] > 32) == (large == 1))
                            S.h_work.push_back(make_int2(i, K));
                }
                const int cnt = (int)(S.h_work.size() - off);
                if (cnt) S.launches.push_back({0, dt, large, off, cnt, -1});
                if (!cnt || !large) continue;
                // Dinv_K of the wide ones, a CTA per 32 x 32 tile of its lower triangle
                // (the LU form's own Dinv comes from k_linv)
                const int64_t off2 = (int64_t)S.h_work.size();
                for (int64_t e = off; e < off + cnt; e++) {
                    const int2 wk = S.h_work[e];
                    if (descs[wk.x].lu) continue;
                    const int s = plans[wk.x]->super_ptr[wk.y + 1] - plans[wk.x]->super_ptr[wk.y];
                    const int nt = (s + 31) / 32;
                    for (int t = 0; t < nt * (nt + 1) / 2; t++) S.h_work.push_back(make_int2(wk.x, (wk.y << 8) | t));
                }
                const int cnt2 = (int)(S.h_work.size() - off2);
                if (cnt2) S.launches.push_back({KL_DINV, dt, 0, off2, cnt2, -1});
            }
        // 2) Lhat for every row tile: the tensor-core product for eligible
        //    supernodes (after the digit planes of L_KK^{-1}), FP64 for the rest
        {
            const int64_t off = (int64_t)S.h_work.size();
            for (int i = 0; i < np; i++) {
                const PlanData &p = *plans[i];
                for (int32_t K = 0; K < p.ns; K++) {
                    const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                    const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
                    if (c == 0 || !actn(i, K) || !ozok(i, s)) continue;
                    // bit 7: the tcgen05 operand layout, for the transposed Lhat product
                    const int tcl = lhat_tc(i, s) ? 0x80 : 0;
                    for (int jb = 0; jb < (s + 7) / 8; jb++) S.h_work.push_back(make_int2(i, (K << 8) | tcl | jb));
                }
            }
            const int cnt = (int)(S.h_work.size() - off);
            if (cnt) S.launches.push_back({KL_LINV_DIGITS, SELINV_F64, 0, off, cnt, -1});
        }
        {
            // Lhat of the supernodes wider than 64 columns on tcgen05: (K, 64-row tile) items
            const int64_t off = (int64_t)S.h_items.size();
            for (int i = 0; i < np; i++) {
                const PlanData &p = *plans[i];
                for (int32_t K = 0; K < p.ns; K++) {
                    const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                    const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
                    if (c == 0 || !actn(i, K) || !ozok(i, s) || !lhat_tc(i, s)) continue;
                    for (int64_t t = 0; t < (c + kTcWideRows - 1) / kTcWideRows; t++) S.h_items.push_back({i, K, (int)t, 1});
                }
            }
            const int cnt = (int)(S.h_items.size() - off);
            if (cnt) S.launches.push_back({KL_LHAT_OZ, SELINV_F64, kTcWide, off, cnt, -1});
        }
        for (int tn : {64, 32, 16}) {
            const int64_t off = (int64_t)S.h_items.size();
            for (int i = 0; i < np; i++) {
                const PlanData &p = *plans[i];
                for (int32_t K = 0; K < p.ns; K++) {
                    const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                    const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
                    if (c == 0 || !actn(i, K) || !ozok(i, s) || lhat_tc(i, s)) continue;
                    const int ktn = s <= 16 ? 16 : 32;   // 32-column tiles: two CTAs per SM
                    if (ktn != tn) continue;
                    const int ncol = (s + tn - 1) / tn;
                    for (int t = 0; t < p.ntiles[K]; t++)
                        for (int ct = 0; ct < ncol; ct++) S.h_items.push_back({i, K, t * ncol + ct, p.ntiles[K]});
                }
            }
            const int cnt = (int)(S.h_items.size() - off);
            if (cnt) S.launches.push_back({KL_LHAT_OZ, SELINV_F64, tn, off, cnt, -1});
        }
        for (int dt = 0; dt < 2; dt++)
            for (int b = 0; b < kNumBuckets; b++) {
                const int64_t off = (int64_t)S.h_items.size();
                for (int i = 0; i < np; i++) {
                    if (descs[i].dtype != dt) continue;
                    const PlanData &p = *plans[i];
                    for (int32_t K = 0; K < p.ns; K++) {
                        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
                        if (c == 0 || !actn(i, K) || bucket_of(s) != b || ozok(i, s)) continue;
                        for (int t = 0; t < p.ntiles[K]; t++) S.h_items.push_back({i, K, t, p.ntiles[K]});
                    }
                }
                const int cnt = (int)(S.h_items.size() - off);
                if (cnt) S.launches.push_back({1, dt, b, off, cnt, -1});
            }
        // 2b) bf16 digit planes of Lhat for the tensor-core contraction
        {
            const int64_t off = (int64_t)S.h_work.size();
            for (int i = 0; i < np; i++) {
                const PlanData &p = *plans[i];
                for (int32_t K = 0; K < p.ns; K++) {
                    const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                    const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
                    if (c == 0 || !actn(i, K) || mode == SELINV_SCHED_PERSISTENT || mode == SELINV_SCHED_PUSH ||
                        !ozok(i, s))
                        continue;
                    // bit 7: only the tcgen05 layout is read (tcgen05 gather-GEMM and
                    // diagonal block); the mma.sync kernels read the other one
                    const int only_u = p.opts.fast_contraction == 1 && s > 32 ? 0x80 : 0;
                    for (int jb = 0; jb < (s + 7) / 8; jb++) S.h_work.push_back(make_int2(i, (K << 8) | only_u | jb));
                }
            }
            const int cnt = (int)(S.h_work.size() - off);
            if (cnt) S.launches.push_back({KL_DIGITS, SELINV_F64, 0, off, cnt, -1});
            // the complex operand (after the FP64 Lhat of step 2)
            const int64_t offz = (int64_t)S.h_work.size();
            for (int i = 0; i < np; i++) {
                const PlanData &p = *plans[i];
                for (int32_t K = 0; K < p.ns; K++) {
                    const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                    const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
                    if (c == 0 || !actn(i, K) || !zok(i, s)) continue;
                    for (int jb = 0; jb < (s + 7) / 8; jb++) S.h_work.push_back(make_int2(i, (K << 8) | jb));
                }
            }
            const int cntz = (int)(S.h_work.size() - offz);
            if (cntz) S.launches.push_back({KL_DIGITS, SELINV_C128, 0, offz, cntz, -1});
        }
        for (size_t q = ph_first; q < S.launches.size(); q++) S.launches[q].side = ph;
    }
    // 3) the traversal, root to leaves
    auto push_items = [&](int i, int32_t K) {
        const PlanData &p = *plans[i];
        for (int t = 0; t < p.ntiles[K]; t++) S.h_items.push_back({i, K, t, p.ntiles[K]});
    };
    // after a tcgen05 launch: the reduction of its split-k row tiles
    auto add_tc_reduce = [&](const Launch tl) {
        const int64_t off = (int64_t)S.h_red.size();
        for (int64_t e = tl.off; e < tl.off + tl.count; e++) {
            const Item &it = S.h_items[e];
            const PlanData &p = *plans[it.prob];
            const int s = p.super_ptr[it.K + 1] - p.super_ptr[it.K];
            const int ncol = tl.bucket == kTcWide ? 1 : (s + tl.bucket - 1) / tl.bucket;
            if (it.ntiles < 2 || it.tile % (it.ntiles * ncol) != 0) continue;   // not a group's first item
            // output rows of the item: s columns, or the 2s (part, column)
            // rows of a complex one in 128-row m tiles
            int rows = s;
            if (tl.bucket == kTcWide && tl.dtype != SELINV_F64) {
                const int nmt = (2 * s + kTcRows - 1) / kTcRows, mt = (it.tile / it.ntiles) % nmt;
                rows = std::min(kTcRows, 2 * s - mt * kTcRows);
            }
            for (int cb = 0; cb < (rows + 7) / 8; cb++) S.h_red.push_back(make_int4((int)e, (int)(e - tl.off), cb, 0));
        }
        const int cnt = (int)((int64_t)S.h_red.size() - off);
        if (cnt) S.launches.push_back({KL_TC_REDUCE, tl.dtype, tl.bucket, off, cnt, tl.level});
    };
    // after a tensor-core diagonal-block launch: its finisher, (K, 8 columns) items
    // (K, 2 columns) items, the digit grid's shift (1: tcgen05 sums, 0:
    // mma.sync sums) in the ntiles field; one launch for the diagonal-block
    // launches of a level
    auto add_diag_fin = [&](const std::vector<std::pair<Launch, int>> &dls) {
        if (dls.empty()) return;
        const int64_t off = (int64_t)S.h_items.size();
        for (const auto &db : dls)
            for (int64_t e = db.first.off; e < db.first.off + db.first.count; e++) {
                const Item it = S.h_items[e];
                if (it.tile != 0) continue;                      // one entry per supernode
                const PlanData &p = *plans[it.prob];
                const int s = p.super_ptr[it.K + 1] - p.super_ptr[it.K];
                for (int cb = 0; cb < (s + 1) / 2; cb++) S.h_items.push_back({it.prob, it.K, cb, db.second});
            }
        const int cnt = (int)((int64_t)S.h_items.size() - off);
        if (cnt) S.launches.push_back({KL_DIAG_FIN, dls[0].first.dtype, 0, off, cnt, dls[0].first.level});
    };
    // tensor-core diagonal block: (64-row tile, 32-column pass) items
    auto push_diag = [&](int i, int32_t K) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int np = (s + kDiagCols - 1) / kDiagCols;
        for (int t = 0; t < p.ntiles[K]; t++)
            for (int jb = 0; jb < np; jb++) S.h_items.push_back({i, K, t * np + jb, p.ntiles[K] * np});
    };
    // tcgen05 diagonal block: (chunk of C rows, column tile of width tn) items,
    // ntiles field = number of chunks; enough chunks for about a CTA per SM over
    // the level (diag_units: the level's column tiles), 8 steps at least
    auto dtc_tn = [](int s) { return s <= 32 ? 32 : 64; };
    auto push_diag_tc = [&](int i, int32_t K, int64_t diag_units) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        const int tn = dtc_tn(s), ncol = (s + tn - 1) / tn;
        const int64_t nsteps = (c + 15) / 16;
        const int64_t target = 152;    // a CTA per SM over the level
        const int64_t want = (target + diag_units - 1) / std::max<int64_t>(diag_units, 1);
        const int nch = (int)std::max<int64_t>(1, std::min(want, (nsteps + 7) / 8));
        for (int ch = 0; ch < nch; ch++)
            for (int ct = 0; ct < ncol; ct++) S.h_items.push_back({i, K, ch * ncol + ct, nch});
    };
    // complex tcgen05 items: the transposed gather-GEMM over (64-row tile, m
    // tile of the 2s output rows, k-range), ntiles = number of k-ranges; the
    // diagonal block over (chunk, column tile, m tile), ntiles = number of chunks
    auto z_nmt = [&](int s) { return (2 * s + kTcRows - 1) / kTcRows; };
    auto z_ctas = [&](int i, int32_t K) -> int64_t {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        return c == 0 ? 0 : (c + kTcWideRows - 1) / kTcWideRows * z_nmt(s);
    };
    auto z_split = [&](int i, int32_t K, int64_t level_ctas) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        const selinv_opts &o = p.opts;
        const int64_t target = (int64_t)o.split_target * 152;
        const int64_t want = (target + level_ctas - 1) / std::max<int64_t>(level_ctas, 1);
        const int64_t maxsplit = std::max<int64_t>(1, ((2 * c + 15) / 16) / o.split_min_steps);
        return (int)std::max<int64_t>(1, std::min(want, maxsplit));
    };
    auto push_z = [&](int i, int32_t K, int nsplit) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        if (c == 0) return;
        const int nmt = z_nmt(s);
        const int64_t nt = (c + kTcWideRows - 1) / kTcWideRows;
        for (int64_t t = 0; t < nt; t++)
            for (int mt = 0; mt < nmt; mt++)
                for (int ks = 0; ks < nsplit; ks++) S.h_items.push_back({i, K, (int)((t * nmt + mt) * nsplit + ks), nsplit});
    };
    auto push_zdiag = [&](int i, int32_t K, int64_t diag_units) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        const int tn = s <= 32 ? 32 : 64, ncol = (s + tn - 1) / tn, nmt = z_nmt(s);
        const int64_t nsteps = (2 * c + 15) / 16;
        const int64_t want = (152 + diag_units - 1) / std::max<int64_t>(diag_units, 1);
        const int nch = (int)std::max<int64_t>(1, std::min(want, (nsteps + 7) / 8));
        for (int ch = 0; ch < nch; ch++)
            for (int ct = 0; ct < ncol; ct++)
                for (int mt = 0; mt < nmt; mt++) S.h_items.push_back({i, K, (ch * ncol + ct) * nmt + mt, nch});
    };
    // the launches of the complex tcgen05 supernodes zs (one level, or one
    // supernode in the plain schedule): contraction, its split-k sums, the
    // diagonal block per column-tile width and its finisher
    auto launch_z = [&](const std::vector<std::pair<int, int32_t>> &zs, int level, int64_t other_ctas) {
        if (zs.empty()) return;
        int64_t ctas = other_ctas;
        for (auto &ik : zs) ctas += z_ctas(ik.first, ik.second);
        const int64_t off = (int64_t)S.h_items.size();
        for (auto &ik : zs) push_z(ik.first, ik.second, z_split(ik.first, ik.second, ctas));
        const int cnt = (int)(S.h_items.size() - off);
        if (cnt) {
            S.launches.push_back({KL_SELINV_TC, SELINV_C128, kTcWide, off, cnt, level});
            add_tc_reduce(S.launches.back());
        }
        int64_t units = 0;
        for (auto &ik : zs) {
            const int s = plans[ik.first]->super_ptr[ik.second + 1] - plans[ik.first]->super_ptr[ik.second];
            const int tn = s <= 32 ? 32 : 64;
            units += (int64_t)((s + tn - 1) / tn) * z_nmt(s);
        }
        for (int tn : {64, 32}) {
            const int64_t off2 = (int64_t)S.h_items.size();
            for (auto &ik : zs) {
                const int s = plans[ik.first]->super_ptr[ik.second + 1] - plans[ik.first]->super_ptr[ik.second];
                if ((s <= 32 ? 32 : 64) == tn) push_zdiag(ik.first, ik.second, units);
            }
            const int cnt2 = (int)(S.h_items.size() - off2);
            if (cnt2) {
                S.launches.push_back({KL_DIAG_TC, SELINV_C128, tn, off2, cnt2, level});
                add_diag_fin({{S.launches.back(), 1}});
            }
        }
    };
    // tensor-core items: (row tile, column tile of width tn, k-range) triples,
    // ntiles field = number of k-ranges; c == 0 has none
    auto oz_tn = [](int s) { return s <= 16 ? 16 : (s <= 32 ? 32 : 64); };
    auto use_tc = [&](int i) { return plans[i]->opts.fast_contraction == 1; };
    // supernodes wider than 64 columns on tcgen05 run the transposed kernel
    // (k_selinv_tcw: all columns of K per CTA, 64 rows of C), launch bucket 128
    auto tc_wide = [&](int i, int s) { return use_tc(i) && s > 64; };
    auto tn_of = [&](int i, int s) { return tc_wide(i, s) ? kTcWide : oz_tn(s); };
    // row tiles of the contraction: 64 rows on mma.sync and on the transposed
    // tcgen05 kernel, 128 on the row-tile tcgen05 kernel
    // the diagonal block of a supernode on the tcgen05 engine runs on tcgen05
    // when it is wider than 32 columns, else on the mma.sync kernel (cheaper per item)
    auto diag_tc = [&](int i, int s) { return use_tc(i) && s > 32; };
    auto row_tiles = [&](int i, int32_t K) -> int64_t {
        const PlanData &p = *plans[i];
        if (!use_tc(i)) return p.ntiles[K];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        if (tc_wide(i, s)) return (c + kTcWideRows - 1) / kTcWideRows;
        return (c + kTcRows - 1) / kTcRows;
    };
    auto push_oz = [&](int i, int32_t K, int tn, int nsplit) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        if (c == 0) return;
        const int ncol = tn == kTcWide ? 1 : (s + tn - 1) / tn;   // the transposed kernel covers all columns
        const int64_t nt = row_tiles(i, K);
        for (int t = 0; t < nt; t++)
            for (int ct = 0; ct < ncol; ct++)
                for (int ks = 0; ks < nsplit; ks++) S.h_items.push_back({i, K, (t * ncol + ct) * nsplit + ks, nsplit});
    };
    // k-split of the contraction: enough CTAs for two per SM on narrow levels,
    // each k-range at least 256 long
    auto oz_split = [&](int i, int32_t K, int64_t level_ctas, int cap = 1 << 30) {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        const selinv_opts &o = p.opts;
        const int64_t target = (int64_t)o.split_target * 152;
        const int64_t want = std::min<int64_t>(cap, (target + level_ctas - 1) / std::max<int64_t>(level_ctas, 1));
        const int64_t maxsplit = std::max<int64_t>(1, ((c + 15) / 16) / o.split_min_steps);
        return (int)std::max<int64_t>(1, std::min(want, maxsplit));
    };
    // steps of the first k-range of K's items under split ns (ranges are
    // whole 128-k chunks; the last one takes the rest)
    auto oz_chunk = [&](int i, int32_t K, int ns) -> int64_t {
        const PlanData &p = *plans[i];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - (p.super_ptr[K + 1] - p.super_ptr[K]);
        const int64_t steps = (c + 15) / 16;
        return ((steps + ns - 1) / ns + kTcChunkSteps - 1) / kTcChunkSteps * kTcChunkSteps;
    };
    auto oz_ctas = [&](int i, int32_t K) -> int64_t {
        const PlanData &p = *plans[i];
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
        if (c == 0) return 0;
        return row_tiles(i, K) * (tc_wide(i, s) ? 1 : (s + oz_tn(s) - 1) / oz_tn(s));
    };
    // k-split cap of a level: the split rule's value or a smaller one when an
    // estimate of the level's makespan prefers it.  The estimate assigns the
    // CTAs, longest first, to the SM that frees first (one CTA per SM), each
    // costing its k16 steps plus a fixed cost, and charges a split level the
    // reduction of its partial sums.
    auto level_split = [&](const std::vector<std::pair<int, int32_t>> &oz, int64_t level_ctas) -> int {
        if (oz.empty() || level_ctas <= 0) return 1;
        constexpr int64_t kCtaCost = 8, kReduceCost = 6;   // in k16 steps
        int smax = 1;
        for (auto &ik : oz) smax = std::max(smax, oz_split(ik.first, ik.second, level_ctas));
        int best = smax;
        int64_t best_t = -1;
        std::vector<std::pair<int64_t, int64_t>> lens;   // (cost, CTAs)
        for (int sg = 1; sg <= smax; sg++) {
            lens.clear();
            bool split = false;
            for (auto &ik : oz) {
                const int ns = oz_split(ik.first, ik.second, level_ctas, sg);
                const PlanData &p = *plans[ik.first];
                const int64_t c = p.rowptr[ik.second + 1] - p.rowptr[ik.second] -
                                  (p.super_ptr[ik.second + 1] - p.super_ptr[ik.second]);
                const int64_t steps = (c + 15) / 16, ch = oz_chunk(ik.first, ik.second, ns);
                const int64_t tiles = oz_ctas(ik.first, ik.second);
                split = split || ns > 1;
                for (int x = 0; x < ns; x++)
                    lens.push_back({std::max<int64_t>(0, std::min(ch, steps - x * ch)) + kCtaCost, tiles});
            }
            std::sort(lens.begin(), lens.end(), [](const std::pair<int64_t, int64_t> &a,
                                                   const std::pair<int64_t, int64_t> &b) { return a.first > b.first; });
            std::vector<int64_t> heap(152, 0);   // min-heap of the SMs' finish times
            for (auto &lc : lens)
                for (int64_t m = 0; m < lc.second; m++) {
                    std::pop_heap(heap.begin(), heap.end(), std::greater<int64_t>());
                    heap.back() += lc.first;
                    std::push_heap(heap.begin(), heap.end(), std::greater<int64_t>());
                }
            const int64_t t = *std::max_element(heap.begin(), heap.end()) + (split ? kReduceCost : 0);
            if (best_t < 0 || t < best_t) {
                best_t = t;
                best = sg;
            }
        }
        return best;
    };

    if (mode == SELINV_SCHED_PERSISTENT) {
        // one persistent launch per element type over every supernode of every
        // problem, root level first (FP64 / complex contraction kernel)
        int nlev = 0;
        for (int i = 0; i < np; i++) nlev = std::max(nlev, plans[i]->nlevels);
        for (int dt = 0; dt < 2; dt++) {
            const int64_t off = (int64_t)S.h_items.size();
            for (int l = 0; l < nlev; l++)
                for (int i = 0; i < np; i++) {
                    if (descs[i].dtype != dt) continue;
                    const PlanData &p = *plans[i];
                    if (l >= p.nlevels) continue;
                    for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++)
                        if (act(i, p.level_list[e])) push_items(i, p.level_list[e]);
                }
            const int cnt = (int)(S.h_items.size() - off);
            S.h_buckets.resize(S.h_items.size());
            for (int64_t e = off; e < (int64_t)S.h_items.size(); e++) {
                const Item &it = S.h_items[e];
                const PlanData &p = *plans[it.prob];
                S.h_buckets[e] = (int8_t)bucket_of(p.super_ptr[it.K + 1] - p.super_ptr[it.K]);
            }
            if (cnt) S.launches.push_back({KL_PERSIST, dt, 0, off, cnt, 0});
        }
    } else if (mode == SELINV_SCHED_PUSH) {
        // Alg. 2, left-looking: per level (root first) the diagonal blocks of its
        // supernodes, then their pushes into the descendants, grouped by the
        // width class of the target
        int nlev = 0;
        for (int i = 0; i < np; i++) nlev = std::max(nlev, plans[i]->nlevels);
        // (I', segment) pairs by the level of the segment's owner
        std::vector<std::vector<std::vector<int2>>> by_level(np);
        for (int i = 0; i < np; i++) {
            const PlanData &p = *plans[i];
            by_level[i].assign(std::max(p.nlevels, 1), {});
            for (int32_t I = 0; I < p.ns; I++) {
                if (!act(i, I)) continue;
                for (int64_t e = p.seg_ptr[I]; e < p.seg_ptr[I + 1]; e++)
                    by_level[i][p.level[p.seg_owner[e]]].push_back(make_int2(I, (int)(e - p.seg_ptr[I])));
            }
        }
        for (int l = 0; l < nlev; l++) {
            for (int dt = 0; dt < 2; dt++)
                for (int b = kNumBuckets - 1; b >= 0; b--) {
                    const int64_t off = (int64_t)S.h_items.size();
                    for (int i = 0; i < np; i++) {
                        if (descs[i].dtype != dt) continue;
                        const PlanData &p = *plans[i];
                        if (l >= p.nlevels) continue;
                        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                            const int32_t K = p.level_list[e];
                            if (act(i, K) && bucket_of(p.super_ptr[K + 1] - p.super_ptr[K]) == b) push_items(i, K);
                        }
                    }
                    const int cnt = (int)(S.h_items.size() - off);
                    if (cnt) S.launches.push_back({KL_PUSH_DIAG, dt, b, off, cnt, l});
                }
            for (int dt = 0; dt < 2; dt++)
                for (int b = kNumBuckets - 1; b >= 0; b--) {
                    const int64_t off = (int64_t)S.h_items.size();
                    for (int i = 0; i < np; i++) {
                        if (descs[i].dtype != dt) continue;
                        const PlanData &p = *plans[i];
                        if (l >= p.nlevels) continue;
                        for (const int2 &pr : by_level[i][l]) {
                            const int32_t I = pr.x;
                            const int s = p.super_ptr[I + 1] - p.super_ptr[I];
                            if (bucket_of(s) != b) continue;
                            const int64_t c = p.rowptr[I + 1] - p.rowptr[I] - s;
                            const int64_t e = p.seg_ptr[I] + pr.y;
                            const int64_t q0 = p.seg_start[e];
                            const int64_t q1 = e + 1 < p.seg_ptr[I + 1] ? p.seg_start[e + 1] : c;
                            for (int64_t t = 0; t < (q1 - q0 + kTM - 1) / kTM; t++)   // inner product rows
                                S.h_items.push_back({i, I, (int)t, (pr.y << 1) | 1});
                            for (int64_t t = 0; t < (c - q1 + kTM - 1) / kTM; t++)    // outer product rows
                                S.h_items.push_back({i, I, (int)t, pr.y << 1});
                        }
                    }
                    const int cnt = (int)(S.h_items.size() - off);
                    if (cnt) S.launches.push_back({KL_PUSH, dt, b, off, cnt, l});
                }
        }
    } else if (mode == SELINV_SCHED_PLAIN) {
        // one launch per supernode, K = N..1, problem after problem
        for (int i = 0; i < np; i++) {
            const PlanData &p = *plans[i];
            for (int32_t K = p.ns - 1; K >= 0; K--) {
                if (!act(i, K)) continue;
                const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                if (zok(i, s)) {
                    launch_z({{i, K}}, p.level[K], 0);
                    continue;
                }
                if (ozok(i, s)) {
                    const int tn = tn_of(i, s);
                    const int64_t off = (int64_t)S.h_items.size();
                    push_oz(i, K, tn, oz_split(i, K, oz_ctas(i, K)));
                    if (S.h_items.size() > (size_t)off) {
                        S.launches.push_back({use_tc(i) ? KL_SELINV_TC : KL_SELINV_OZ, descs[i].dtype, tn, off,
                                              (int)(S.h_items.size() - off), p.level[K]});
                        if (use_tc(i)) add_tc_reduce(S.launches.back());
                    }
                    const int64_t off2 = (int64_t)S.h_items.size();
                    if (diag_tc(i, s)) {
                        push_diag_tc(i, K, (s + dtc_tn(s) - 1) / dtc_tn(s));
                        S.launches.push_back({KL_DIAG_TC, descs[i].dtype, dtc_tn(s), off2,
                                              (int)(S.h_items.size() - off2), p.level[K]});
                        add_diag_fin({{S.launches.back(), 1}});
                    } else {
                        push_diag(i, K);
                        S.launches.push_back({KL_DIAG, descs[i].dtype, bucket_of(s), off2,
                                              (int)(S.h_items.size() - off2), p.level[K]});
                        add_diag_fin({{S.launches.back(), 0}});
                    }
                    continue;
                }
                const int64_t off = (int64_t)S.h_items.size();
                push_items(i, K);
                S.launches.push_back({KL_SELINV, descs[i].dtype, bucket_of(s), off,
                                      (int)(S.h_items.size() - off), p.level[K]});
            }
        }
    } else {
        int nlev = 0;
        for (int i = 0; i < np; i++) nlev = std::max(nlev, plans[i]->nlevels);
        for (int l = 0; l < nlev; l++) {
            if (nph >= 2 && l == ltop) S.join_at = (int)S.launches.size();
            if (nph == 3 && l == lmid) S.join_at2 = (int)S.launches.size();
            // tensor-core contraction of every eligible supernode of the level
            // (one launch per column-tile width), then their diagonal blocks
            std::vector<std::pair<int, int32_t>> oz;  // (problem, K)
            for (int i = 0; i < np; i++) {
                const PlanData &p = *plans[i];
                if (l >= p.nlevels) continue;
                for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                    const int32_t K = p.level_list[e];
                    if (act(i, K) && ozok(i, p.super_ptr[K + 1] - p.super_ptr[K]))
                        oz.push_back({i, K});
                }
            }
            std::vector<std::pair<int, int32_t>> zs;   // complex tcgen05 supernodes of the level
            for (int i = 0; i < np; i++) {
                const PlanData &p = *plans[i];
                if (l >= p.nlevels) continue;
                for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                    const int32_t K = p.level_list[e];
                    if (act(i, K) && zok(i, p.super_ptr[K + 1] - p.super_ptr[K])) zs.push_back({i, K});
                }
            }
            int64_t level_ctas = 0;
            for (auto &ik : oz) level_ctas += oz_ctas(ik.first, ik.second);
            launch_z(zs, l, level_ctas);
            // the level's split, and its supernodes in the order of their items'
            // length, longest first (the CTAs that start last are short ones)
            const int sig = level_split(oz, level_ctas);
            std::stable_sort(oz.begin(), oz.end(), [&](const std::pair<int, int32_t> &a, const std::pair<int, int32_t> &b) {
                return oz_chunk(a.first, a.second, oz_split(a.first, a.second, level_ctas, sig)) >
                       oz_chunk(b.first, b.second, oz_split(b.first, b.second, level_ctas, sig));
            });
            for (int tc = 1; tc >= 0; tc--)
                for (int tn : {kTcWide, 64, 32, 16}) {
                    const int64_t off = (int64_t)S.h_items.size();
                    for (auto &ik : oz) {
                        const PlanData &p = *plans[ik.first];
                        const int s = p.super_ptr[ik.second + 1] - p.super_ptr[ik.second];
                        if (tn_of(ik.first, s) == tn && use_tc(ik.first) == (tc == 1))
                            push_oz(ik.first, ik.second, tn, oz_split(ik.first, ik.second, level_ctas, sig));
                    }
                    const int cnt = (int)(S.h_items.size() - off);
                    if (cnt) {
                        S.launches.push_back({tc ? KL_SELINV_TC : KL_SELINV_OZ, SELINV_F64, tn, off, cnt, l});
                        if (tc) add_tc_reduce(S.launches.back());
                    }
                }
            {
                // diagonal blocks: tcgen05 (per column-tile width) or mma.sync
                int64_t diag_units = 0;
                for (auto &ik : oz) {
                    const int s = plans[ik.first]->super_ptr[ik.second + 1] - plans[ik.first]->super_ptr[ik.second];
                    if (diag_tc(ik.first, s)) diag_units += (s + dtc_tn(s) - 1) / dtc_tn(s);
                }
                std::vector<std::pair<Launch, int>> fins;
                for (int tn : {64, 32}) {
                    const int64_t off = (int64_t)S.h_items.size();
                    for (auto &ik : oz) {
                        const int s = plans[ik.first]->super_ptr[ik.second + 1] - plans[ik.first]->super_ptr[ik.second];
                        if (diag_tc(ik.first, s) && dtc_tn(s) == tn) push_diag_tc(ik.first, ik.second, diag_units);
                    }
                    const int cnt = (int)(S.h_items.size() - off);
                    if (cnt) {
                        S.launches.push_back({KL_DIAG_TC, SELINV_F64, tn, off, cnt, l});
                        fins.push_back({S.launches.back(), 1});
                    }
                }
                const int64_t off = (int64_t)S.h_items.size();
                for (auto &ik : oz) {
                    const int s = plans[ik.first]->super_ptr[ik.second + 1] - plans[ik.first]->super_ptr[ik.second];
                    if (!diag_tc(ik.first, s)) push_diag(ik.first, ik.second);
                }
                const int cnt = (int)(S.h_items.size() - off);
                if (cnt) {
                    S.launches.push_back({KL_DIAG, SELINV_F64, 0, off, cnt, l});
                    fins.push_back({S.launches.back(), 0});
                }
                add_diag_fin(fins);
            }
            // fused DFMA kernel for everything else: a warp per tiny supernode,
            // a CTA per row tile for the rest
            for (int dt = 0; dt < 2; dt++) {
                const int64_t off = (int64_t)S.h_items.size();
                for (int i = 0; i < np; i++) {
                    if (descs[i].dtype != dt) continue;
                    const PlanData &p = *plans[i];
                    if (l >= p.nlevels) continue;
                    for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                        const int32_t K = p.level_list[e];
                        if (act(i, K) && tiny(i, K)) S.h_items.push_back({i, K, 0, 1});
                    }
                }
                const int cnt = (int)(S.h_items.size() - off);
                if (cnt) S.launches.push_back({KL_SELINV_TINY, dt, 0, off, cnt, l});
            }
            for (int dt = 0; dt < 2; dt++)
                for (int b = kNumBuckets - 1; b >= 0; b--) {
                    const int64_t off = (int64_t)S.h_items.size();
                    for (int i = 0; i < np; i++) {
                        if (descs[i].dtype != dt) continue;
                        const PlanData &p = *plans[i];
                        if (l >= p.nlevels) continue;
                        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                            const int32_t K = p.level_list[e];
                            const int s = p.super_ptr[K + 1] - p.super_ptr[K];
                            if (act(i, K) && bucket_of(s) == b && !ozok(i, s) && !zok(i, s) && !tiny(i, K))
                                push_items(i, K);
                        }
                    }
                    const int cnt = (int)(S.h_items.size() - off);
                    if (cnt) S.launches.push_back({KL_SELINV, dt, b, off, cnt, l});
                }
        }
    }
    S.h_descs = descs;
    int rc;
    if ((rc = upload(&S.d_descs, S.h_descs))) return rc;
    if ((rc = upload(&S.d_items, S.h_items))) return rc;
    if ((rc = upload(&S.d_work, S.h_work))) return rc;
    if (!S.h_buckets.empty() && (rc = upload(&S.d_buckets, S.h_buckets))) return rc;
    // the exact diagonal-block sums and the column maxima of A^{-1}_{C,K} start
    // from zero in every call
    {
        std::vector<char> has(np, 0);
        for (const Launch &L : S.launches)
            if (L.kind == KL_DIAG || L.kind == KL_DIAG_TC)
                for (int64_t e = L.off; e < L.off + L.count; e++) has[S.h_items[e].prob] = 1;
        for (int i = 0; i < np; i++) {
            if (!has[i]) continue;
            S.pre_ptr.push_back(descs[i].dacc);
            S.pre_bytes.push_back(sizeof(long long) * (descs[i].dtype == SELINV_F64 ? 2 : 4) *
                                  (size_t)std::max<int64_t>(plans[i]->linv_total, 1));
            S.pre_ptr.push_back(descs[i].colexpY);
            S.pre_bytes.push_back(sizeof(int) * (size_t)std::max(plans[i]->n, 1));
        }
    }
    // the push schedule accumulates into A^{-1}: zero at the start of every call
    if (mode == SELINV_SCHED_PUSH)
        for (int i = 0; i < np; i++) {
            S.pre_ptr.push_back(descs[i].Z);
            S.pre_bytes.push_back(elem_size(descs[i].dtype) * (size_t)std::max<int64_t>(plans[i]->nnz, 1));
        }
    // one partial (hi, lo) tile of 128 x 64 per CTA of the widest tcgen05 launch
    int64_t tc_ctas = 0;
    for (const Launch &L : S.launches)
        if (L.kind == KL_SELINV_TC) tc_ctas = std::max<int64_t>(tc_ctas, L.count);
    if (tc_ctas > 0 &&
        cudaMalloc((void **)&S.tcslab, sizeof(long long) * (size_t)kTcSlotWords * (size_t)tc_ctas) != cudaSuccess)
        return SELINV_ERR_OOM;

    if (!S.h_red.empty() && (rc = upload(&S.d_red, S.h_red))) return rc;
    return SELINV_OK;
}

// one launch of a schedule with the problem descriptors at `d`
cudaError_t launch_with(const Schedule &S, const Launch &L, const ProbDesc *d, cudaStream_t st) {
    switch (L.kind) {
    // the wide supernodes' Dinv follows in KL_DINV launches (32 x 32 tiles)
    case KL_LINV: return launch_linv(L.dtype, d, S.d_work + L.off, L.count, L.bucket, st, L.bucket == 0);
    case KL_DINV: return launch_dinv(L.dtype, d, S.d_work + L.off, L.count, st);
    case KL_LHAT: return launch_lhat(L.dtype, L.bucket, d, S.d_items + L.off, L.count, st);
    case KL_SELINV: return launch_selinv(L.dtype, L.bucket, d, S.d_items + L.off, L.count, st);
    case KL_DIGITS:
        if (L.dtype != SELINV_F64) return launch_lhat_digits_z(d, S.d_work + L.off, L.count, st);
        return launch_lhat_digits(d, S.d_work + L.off, L.count, st);
    case KL_SELINV_OZ: return launch_selinv_oz(L.bucket, d, S.d_items + L.off, L.count, st);
    case KL_DIAG: return launch_diag_oz(d, S.d_items + L.off, L.count, st);
    case KL_LINV_DIGITS: return launch_linv_digits(d, S.d_work + L.off, L.count, st);
    case KL_LHAT_OZ:
        if (L.bucket == kTcWide) return launch_lhat_tcw(d, S.d_items + L.off, L.count, S.spin_limit, st);
        return launch_lhat_oz(L.bucket, d, S.d_items + L.off, L.count, st);
    case KL_SELINV_TC:
        if (L.bucket == kTcWide)
            return launch_selinv_tcw(L.dtype != SELINV_F64, d, S.d_items + L.off, L.count, S.tcslab, S.spin_limit, st);
        return launch_selinv_tc(L.bucket, d, S.d_items + L.off, L.count, S.tcslab, S.spin_limit, st);
    case KL_TC_REDUCE:
        if (L.bucket == kTcWide)
            return launch_tcw_reduce(L.dtype != SELINV_F64, d, S.d_items, S.d_red + L.off, L.count, S.tcslab, st);
        return launch_tc_reduce(L.bucket, d, S.d_items, S.d_red + L.off, L.count, S.tcslab, st);
    case KL_DIAG_FIN:
        if (L.dtype != SELINV_F64) return launch_diag_fin_z(d, S.d_items + L.off, L.count, st);
        return launch_diag_fin(d, S.d_items + L.off, L.count, st);
    case KL_DIAG_TC:
        return launch_diag_tc(L.bucket, L.dtype != SELINV_F64, d, S.d_items + L.off, L.count, S.spin_limit, st);
    case KL_SELINV_TINY: return launch_selinv_tiny(L.dtype, d, S.d_items + L.off, L.count, st);
    case KL_PUSH_DIAG: return launch_push(L.dtype, 0, L.bucket, d, S.d_items + L.off, L.count, st);
    case KL_PUSH: return launch_push(L.dtype, 1, L.bucket, d, S.d_items + L.off, L.count, st);
    case KL_PERSIST: {
        for (size_t r = 0; r < S.reset_ptr.size(); r++) {
            cudaError_t e = cudaMemsetAsync(S.reset_ptr[r], 0, S.reset_bytes[r], st);
            if (e != cudaSuccess) return e;
        }
        return launch_selinv_persist(L.dtype, d, S.d_items + L.off, S.d_buckets + L.off, L.count,
                                     S.ticket, S.spin_limit, S.wait_on_unset, st);
    }
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_one(const Schedule &S, const Launch &L, cudaStream_t st) { return launch_with(S, L, S.d_descs, st); }

static cudaError_t issue_pre(const Schedule &S, cudaStream_t st) {
    for (size_t r = 0; r < S.pre_ptr.size(); r++) {
        cudaError_t e = cudaMemsetAsync(S.pre_ptr[r], 0, S.pre_bytes[r], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

const char *launch_kind_name(int kind) {
    static const char *names[KL_NKINDS] = {"linv", "lhat", "selinv", "lhat_digits", "selinv_oz", "diag",
                                           "linv_digits", "lhat_oz", "persist", "selinv_tc", "tc_reduce",
                                           "diag_fin", "push_diag", "push", "dinv", "diag_tc", "selinv_tiny"};
    return kind >= 0 && kind < KL_NKINDS ? names[kind] : "?";
}

// Optional additions of a host-buffer call to the issue of a schedule: an
// event the side stream waits for at its fork (the inputs it reads have
// landed), and callbacks run before given launches (at the end for index
// == the number of launches), in ascending order.
struct IssueHooks {
    cudaEvent_t side_wait[2] = {nullptr, nullptr};   // before the side stream's first / second phase
    std::vector<int> mark_at;
    std::function<cudaError_t(int)> mark;
};

// The launches in order on `st`, those marked `side` on the schedule's side
// stream: it forks from `st` at its first launch and joins back before launch
// join_at (or at the end).
static cudaError_t issue(Schedule &S, cudaStream_t st, bool count, const IssueHooks *hk = nullptr) {
    if (count) note_launch((int)S.launches.size());
    cudaError_t e0 = issue_pre(S, st);
    if (e0 != cudaSuccess) return e0;
    bool forked = false;
    auto join = [&]() -> cudaError_t {
        forked = false;
        cudaError_t e = cudaEventRecord(S.ev_join, S.side);
        return e == cudaSuccess ? cudaStreamWaitEvent(st, S.ev_join, 0) : e;
    };
    size_t g = 0;   // next hook mark
    auto marks = [&](size_t i) -> cudaError_t {
        for (; hk && g < hk->mark_at.size() && hk->mark_at[g] == (int)i; g++) {
            const cudaError_t e = hk->mark((int)g);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    int side_phase = 0;   // phase of the side stream's last launch
    for (size_t i = 0; i < S.launches.size(); i++) {
        const Launch &L = S.launches[i];
        cudaError_t e = marks(i);
        if (e != cudaSuccess) return e;
        if (forked && (int)i == S.join_at) {
            if (S.join_at2 < 0) e = join();   // (two phases: the side stream's whole work)
            else e = cudaStreamWaitEvent(st, S.ev_mid, 0);
            if (e != cudaSuccess) return e;
        }
        if (forked && (int)i == S.join_at2 && (e = join()) != cudaSuccess) return e;
        cudaStream_t ls = st;
        if (L.side) {
            if (!forked) {
                if (!S.side && (e = cudaStreamCreateWithFlags(&S.side, cudaStreamNonBlocking)) != cudaSuccess) return e;
                for (cudaEvent_t *ev : {&S.ev_fork, &S.ev_join, &S.ev_mid})
                    if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
                if ((e = cudaEventRecord(S.ev_fork, st)) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(S.side, S.ev_fork, 0)) != cudaSuccess) return e;
                forked = true;
            }
            if (L.side != side_phase) {   // the side stream enters a phase
                if (side_phase == 1 && (e = cudaEventRecord(S.ev_mid, S.side)) != cudaSuccess) return e;
                cudaEvent_t w = hk && L.side <= 2 ? hk->side_wait[L.side - 1] : nullptr;
                if (w && (e = cudaStreamWaitEvent(S.side, w, 0)) != cudaSuccess) return e;
                side_phase = L.side;
            }
            ls = S.side;
        }
        char name[48];
        std::snprintf(name, sizeof(name), "L%d %s", L.level, launch_kind_name(L.kind));
        NvtxRange r(name);
        if ((e = launch_one(S, L, ls)) != cudaSuccess) return e;
    }
    if (forked) {
        const cudaError_t e = join();
        if (e != cudaSuccess) return e;
    }
    return marks(S.launches.size());
}

// The kernel-to-kernel edges of a captured level loop become programmatic
// ones on the programmatic port: the next grid is scheduled as the blocks of
// the previous one finish (none triggers earlier), without the full
// serialization of an ordinary edge, and each kernel waits in
// grid_dep_wait() for its predecessors to complete.  Edges into or out of
// other nodes (copies, memsets) stay full dependencies.  An edge that cannot
// be converted stays as it was; the result is an error only when an edge
// could be neither converted nor restored (the graph must then be dropped).
cudaError_t programmatic_edges(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return cudaSuccess;
    }
    std::vector<cudaGraphNode_t> from(n), to(n);
    std::vector<cudaGraphEdgeData> ed(n);
    if (cudaGraphGetEdges(g, from.data(), to.data(), ed.data(), &n) != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    for (size_t i = 0; i < n; i++) {
        cudaGraphNodeType ta, tb;
        if (cudaGraphNodeGetType(from[i], &ta) != cudaSuccess || cudaGraphNodeGetType(to[i], &tb) != cudaSuccess ||
            ta != cudaGraphNodeTypeKernel || tb != cudaGraphNodeTypeKernel || ed[i].type != cudaGraphDependencyTypeDefault)
            continue;
        cudaGraphEdgeData pe;
        std::memset(&pe, 0, sizeof(pe));
        pe.from_port = cudaGraphKernelNodePortProgrammatic;
        pe.type = cudaGraphDependencyTypeProgrammatic;
        if (cudaGraphRemoveDependencies(g, &from[i], &to[i], &ed[i], 1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (cudaGraphAddDependencies(g, &from[i], &to[i], &pe, 1) != cudaSuccess) {
            cudaGetLastError();
            const cudaError_t e = cudaGraphAddDependencies(g, &from[i], &to[i], &ed[i], 1);
            if (e != cudaSuccess) return e;
        }
    }
    cudaGetLastError();
    return cudaSuccess;
}

int run_schedule(Schedule &S, cudaStream_t st, bool use_graph) {
    // graphs need a capturable stream (not the legacy default stream)
    if (use_graph && st != nullptr && st != cudaStreamLegacy) {
        if (!S.graph) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SELINV_ERR_CUDA;
            cudaError_t e = issue(S, st, false);
            cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return SELINV_ERR_CUDA;
            }
            if (programmatic_edges(g) != cudaSuccess) {
                cudaGraphDestroy(g);
                return SELINV_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&S.graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                S.graph = nullptr;
                return SELINV_ERR_CUDA;
            }
        }
        note_launch((int)S.launches.size());
        return cudaGraphLaunch(S.graph, st) == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
    }
    return issue(S, st, true) == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}

}  // namespace selinv

using namespace selinv;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static bool opts_valid(const selinv_opts *o) {
    return o->schedule >= 0 && o->schedule <= 3 && o->fast_contraction >= 0 && o->fast_contraction <= 2 &&
           o->split_target >= 1 && o->split_target <= 8 && o->split_min_steps >= 8 &&
           o->split_min_steps <= 64 && o->split_min_steps % 8 == 0 && o->oz_min_s >= kOzMinS && o->oz_min_s <= 128 &&
           o->spin_limit > 0 && o->debug_checks >= 0 && o->debug_checks <= 7;
}

extern "C" void selinv_default_opts(selinv_opts *o) {
    if (!o) return;
    o->symmetrize = 1;
    o->schedule = SELINV_SCHED_LEVEL;
    o->autotune = 0;
    o->debug_checks = 0;
    o->spin_limit = 1LL << 22;   // about a second of 256 ns polls
    o->use_graph = 1;
    o->fast_contraction = 1;
    o->split_target = 2;
    o->split_min_steps = 16;
    o->oz_min_s = 16;
}

extern "C" int selinv_symbolic(int32_t n, int32_t nsuper, const int32_t *super_ptr,
                               const int32_t *sparent, const int64_t *rowptr, const int32_t *rowind,
                               const selinv_opts *opts, selinv_plan *out_plan) {
    NvtxRange nvtx_range("selinv_symbolic");
    if (!out_plan) return SELINV_ERR_INVALID_ARG;
    *out_plan = nullptr;
    if (n < 0 || nsuper < 0 || (nsuper == 0) != (n == 0) || !super_ptr || !rowptr ||
        (nsuper > 0 && (!sparent || !rowind)))
        return SELINV_ERR_INVALID_ARG;
    selinv_plan_s *pl = new (std::nothrow) selinv_plan_s();
    if (!pl) return SELINV_ERR_OOM;
    if (opts) {
        if (!opts_valid(opts)) {
            delete pl;
            return SELINV_ERR_INVALID_ARG;
        }
        pl->data.opts = *opts;
    } else {
        selinv_default_opts(&pl->data.opts);
    }
    int rc;
    try {
        rc = build_plan(pl->data, n, nsuper, super_ptr, sparent, rowptr, rowind);
    } catch (const std::bad_alloc &) {
        rc = SELINV_ERR_OOM;
    }
    if (rc != SELINV_OK) {
        selinv_plan_destroy(pl);
        return rc;
    }
    *out_plan = pl;
    return SELINV_OK;
}

selinv_plan_s::~selinv_plan_s() {
    DeviceGuard g(data.device);   // free on the plan's device, whichever is current
    single.release();
    lu.release();
    host.release();
    for (auto &b : batch_cache) b.sched.release();
    for (auto &w : ws) w.release();
    factor_release(this);
    data.release_device();
}

extern "C" void selinv_plan_destroy(selinv_plan plan) { delete plan; }

extern "C" int64_t selinv_plan_nnz(selinv_plan plan) { return plan ? plan->data.nnz : SELINV_ERR_INVALID_ARG; }

extern "C" int64_t selinv_plan_panel_offset(selinv_plan plan, int32_t K) {
    if (!plan || K < 0 || K > plan->data.ns) return -1;
    return plan->data.panel_off[K];
}

extern "C" int selinv_plan_stats(selinv_plan plan, selinv_dtype dtype, double *flops, double *bytes) {
    if (!plan) return SELINV_ERR_INVALID_ARG;
    const PlanData &p = plan->data;
    double F = 0, B = 0;
    const double w = dtype == SELINV_F64 ? 8.0 : 16.0;
    for (int32_t K = 0; K < p.ns; K++) {
        const double s = p.super_ptr[K + 1] - p.super_ptr[K];
        const double c = (double)(p.rowptr[K + 1] - p.rowptr[K]) - s;
        F += 2 * c * c * s + 2 * c * s * s + c * s * s + s * s * s;
        B += w * (c * (c + 1) / 2 + 2 * (c + s) * s + s);
    }
    if (dtype != SELINV_F64) F *= 4;
    if (flops) *flops = F;
    if (bytes) *bytes = B;
    return SELINV_OK;
}

extern "C" int64_t selinv_plan_get(selinv_plan plan, int field, void *dst) {
    if (!plan) return SELINV_ERR_INVALID_ARG;
    const PlanData &p = plan->data;
    const void *src = nullptr;
    int64_t cnt = 0;
    size_t es = 4;
    switch (field) {
    case 0: src = p.level.data(); cnt = p.ns; break;
    case 1: src = p.seg_ptr.data(); cnt = p.ns + 1; es = 8; break;
    case 2: src = p.seg_owner.data(); cnt = (int64_t)p.seg_owner.size(); break;
    case 3: src = p.seg_start.data(); cnt = (int64_t)p.seg_start.size(); break;
    case 4: src = p.seg_coloff.data(); cnt = (int64_t)p.seg_coloff.size(); break;
    case 5: src = p.rel_ptr.data(); cnt = (int64_t)p.rel_ptr.size(); es = 8; break;
    case 6: src = p.relidx.data(); cnt = (int64_t)p.relidx.size(); break;
    case 7: src = p.level_ptr.data(); cnt = (int64_t)p.level_ptr.size(); es = 8; break;
    case 8: src = p.level_list.data(); cnt = p.ns; break;
    case 9: src = p.panel_off.data(); cnt = p.ns + 1; es = 8; break;
    case 11: src = p.colbase.data(); cnt = p.rowptr[p.ns]; es = 8; break;
    case 12: src = p.relbase.data(); cnt = p.rowptr[p.ns]; es = 8; break;
    case 10: {   // supernodes that run under the current selection (1 = runs)
        if (dst)
            for (int32_t K = 0; K < p.ns; K++)
                static_cast<int32_t *>(dst)[K] = p.active.empty() ? 1 : (int32_t)p.active[K];
        return p.ns;
    }
    default: return SELINV_ERR_INVALID_ARG;
    }
    if (dst && cnt > 0) std::memcpy(dst, src, es * (size_t)cnt);
    return cnt;
}


extern "C" int selinv_plan_get_opts(selinv_plan plan, selinv_opts *opts) {
    if (!plan || !opts) return SELINV_ERR_INVALID_ARG;
    *opts = plan->data.opts;
    return SELINV_OK;
}

extern "C" int selinv_plan_set_opts(selinv_plan plan, const selinv_opts *opts) {
    if (!plan || !opts || !opts_valid(opts)) return SELINV_ERR_INVALID_ARG;
    plan->data.opts = *opts;
    plan->data.tuned[0] = plan->data.tuned[1] = false;
    plan->single.release();
    plan->single.valid = false;
    for (auto &b : plan->batch_cache) b.sched.release();
    plan->batch_cache.clear();
    return SELINV_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static int numeric_run(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D, void *Z,
                       cudaStream_t st);

// Autotuner: coordinate search over the tensor engine, the k-split of narrow
// levels and the narrowest tensor-core supernode, each candidate timed with
// CUDA events on the caller's stream and data (best of two runs after a
// warm-up that builds its schedule); the fastest options stay with the plan.
static int autotune(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D, void *Z,
                    cudaStream_t st) {
    PlanData &p = plan->data;
    p.tuned[dtype] = true;
    if (dtype != SELINV_F64) return SELINV_OK;   // the complex path has no tensor-core variants
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SELINV_ERR_CUDA;
    auto measure = [&](const selinv_opts &o, float *ms) -> int {
        p.opts = o;
        plan->single.release();
        plan->single.valid = false;
        int rc = numeric_run(plan, dtype, L, D, Z, st);
        if (rc) return rc;
        float best = 1e30f;
        for (int r = 0; r < 2; r++) {
            cudaEventRecord(e0, st);
            if ((rc = numeric_run(plan, dtype, L, D, Z, st))) return rc;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return SELINV_ERR_CUDA;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
        *ms = best;
        return SELINV_OK;
    };
    selinv_opts best = p.opts;
    float best_ms = 1e30f;
    int rc = SELINV_OK;
    auto consider = [&](selinv_opts o) {
        if (rc) return;
        float ms;
        rc = measure(o, &ms);
        if (!rc && ms < best_ms) { best_ms = ms; best = o; }
    };
    for (int eng : {1, 2, 0}) {
        selinv_opts o = best;
        o.fast_contraction = eng;
        consider(o);
    }
    if (best.fast_contraction != 0) {
        const selinv_opts e = best;
        for (int tgt : {1, 2, 4})
            for (int mins : {8, 16, 32}) {
                selinv_opts o = e;
                o.split_target = tgt;
                o.split_min_steps = mins;
                consider(o);
            }
        const selinv_opts f = best;
        for (int ozm : {1, 8, 16, 32, 64}) {
            selinv_opts o = f;
            o.oz_min_s = ozm;
            consider(o);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p.opts = best;
    plan->single.release();
    plan->single.valid = false;
    return rc;
}

extern "C" int selinv_numeric(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D,
                              void *Z, void *stream) {
    NvtxRange nvtx_range("selinv_numeric");
    if (!plan || (dtype != SELINV_F64 && dtype != SELINV_C128 && dtype != SELINV_C128H)) return SELINV_ERR_INVALID_ARG;
    PlanData &p = plan->data;
    if (p.ns == 0) return SELINV_OK;
    if (!L || !D || !Z || !aligned16(L) || !aligned16(D) || !aligned16(Z)) return SELINV_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p.opts.autotune && !p.tuned[dtype]) {
        const int rc = autotune(plan, dtype, L, D, Z, st);
        if (rc) return rc;
    }
    return numeric_run(plan, dtype, L, D, Z, st);
}

static int numeric_prepare(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D, void *Z,
                           cudaStream_t st);

static int numeric_run(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D, void *Z,
                       cudaStream_t st) {
    const int rc = numeric_prepare(plan, dtype, L, D, Z, st);
    return rc ? rc : run_schedule(plan->single, st, plan->data.opts.use_graph != 0);
}

// The plan's schedule for (dtype, buffers), built or re-keyed, and the debug
// scan of the inputs; nothing of the selected inversion is issued yet.
static int numeric_prepare(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D, void *Z,
                           cudaStream_t st) {
    PlanData &p = plan->data;
    int rc = ensure_device(p);
    if (rc) return rc;
    if (plan->ws.empty()) plan->ws.resize(1);
    rc = plan->ws[0].ensure(p, dtype);
    if (rc) return rc;
    Schedule &S = plan->single;
    const int mode = p.opts.schedule;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = st != nullptr && st != cudaStreamLegacy &&
                           (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone);
    cudaGetLastError();
    if (S.valid && S.key_dtype == dtype && S.mode == mode && !capturing &&
        (S.key_L != L || S.key_D != D || S.key_Z != Z)) {
        // only the caller's buffers changed: every kernel of the schedule
        // reads them through the device descriptors, so those are rewritten
        // in stream order and the schedule (and its graph) stays
        S.h_descs.assign(1, make_desc(p, plan->ws[0], dtype, L, D, Z, mode == SELINV_SCHED_PERSISTENT));
        if (cudaMemcpyAsync(S.d_descs, S.h_descs.data(), sizeof(ProbDesc), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SELINV_ERR_CUDA;
        S.key_L = L; S.key_D = D; S.key_Z = Z;
    }
    if (!S.valid || S.key_L != L || S.key_D != D || S.key_Z != Z || S.key_dtype != dtype ||
        S.mode != mode) {
        std::vector<const PlanData *> plans{&p};
        const bool persist = mode == SELINV_SCHED_PERSISTENT;
        if (persist && (rc = plan->ws[0].ensure_persistent(p))) return rc;
        std::vector<ProbDesc> descs{make_desc(p, plan->ws[0], dtype, L, D, Z, persist)};
        rc = build_schedule(S, plans, descs, mode);
        if (rc) { S.valid = false; return rc; }
        S.reset_ptr.clear(); S.reset_bytes.clear();
        S.spin_limit = p.opts.spin_limit;
        if (persist) {
            S.ticket = plan->ws[0].ticket;
            S.wait_on_unset = (p.opts.debug_checks & 2) ? 1 : 0;
            S.reset_ptr = {plan->ws[0].done, plan->ws[0].ticket};
            S.reset_bytes = {sizeof(int) * (size_t)(p.ns + 1), sizeof(int)};
        }
        S.valid = true;
        S.key_L = L; S.key_D = D; S.key_Z = Z; S.key_dtype = dtype; S.mode = mode;
    }
    plan->last_stream = st;
    if (p.opts.debug_checks & 1) {
        const int64_t w = dtype == SELINV_F64 ? 1 : 2;
        if (launch_check_finite(L, w * p.nnz, p.d_status, st) != cudaSuccess ||
            launch_check_finite(D, w * p.n, p.d_status, st) != cudaSuccess)
            return SELINV_ERR_CUDA;
        note_launch(2);
    }
    return SELINV_OK;
}

// ---------------------------------------------------------------------------
// Selected inversion from host buffers, the copies overlapped with the
// traversal (level schedule with the side-stream normalization):
//   H2D on one copy stream: D, the panels of the top levels' supernodes
//   (the main stream waits for these), then those of the side stream's
//   first and second normalization phases (each phase waits for its own);
//   D2H on another copy stream: the panels of A^{-1} in groups of levels, each
//   group as soon as the main stream has passed its last level (a panel of
//   A^{-1} is final once its level is done: later levels only read it): the
//   top levels at the join, then levels up to about half and four fifths of
//   the rest's bytes, then the rest; the main stream waits for the last copy.
// Panel ranges are the runs of consecutive supernodes of a group.  With
// pinned host buffers the call is captured once per set of buffers into a
// graph (its copy nodes included) and replayed.  Other schedules, and calls
// that autotune or scan their inputs, copy everything in, run and copy
// everything out on the stream.
// ---------------------------------------------------------------------------
static cudaError_t host_pipe_init(HostPipe &h) {
    cudaError_t e = cudaSuccess;
    if (!h.cin && (e = cudaStreamCreateWithFlags(&h.cin, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if (!h.cout && (e = cudaStreamCreateWithFlags(&h.cout, cudaStreamNonBlocking)) != cudaSuccess) return e;
    for (cudaEvent_t *ev : {&h.ev_top, &h.ev_mid, &h.ev_rest, &h.ev_done, &h.ev_in_done})
        if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    while (h.ev_grp.size() < 4) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
        h.ev_grp.push_back(ev);
    }
    return cudaSuccess;
}

void HostPipe::release() {
    if (cin) cudaStreamDestroy(cin);
    if (cout) cudaStreamDestroy(cout);
    for (cudaEvent_t ev : {ev_top, ev_mid, ev_rest, ev_done, ev_in_done})
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : ev_grp) cudaEventDestroy(ev);
    cin = cout = nullptr;
    ev_top = ev_mid = ev_rest = ev_done = ev_in_done = nullptr;
    ev_grp.clear();
}

extern "C" int selinv_numeric_host(selinv_plan plan, selinv_dtype dtype, const void *L_host, const void *D_host,
                                   void *Ainv_host, void *L_dev, void *D_dev, void *Ainv_dev, void *stream) {
    NvtxRange nvtx_range("selinv_numeric_host");
    if (!plan || (dtype != SELINV_F64 && dtype != SELINV_C128 && dtype != SELINV_C128H)) return SELINV_ERR_INVALID_ARG;
    PlanData &p = plan->data;
    if (p.ns == 0) return SELINV_OK;
    if (!L_host || !D_host || !Ainv_host || !L_dev || !D_dev || !Ainv_dev || !aligned16(L_dev) ||
        !aligned16(D_dev) || !aligned16(Ainv_dev))
        return SELINV_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st != nullptr && st != cudaStreamLegacy &&
        (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone))
        return SELINV_ERR_INVALID_ARG;   // host copies per call: not for a captured stream
    const size_t es = elem_size(dtype);
    const size_t lbytes = es * (size_t)p.nnz, dbytes = es * (size_t)p.n;
    auto whole = [&]() -> int {   // copy in, run, copy out, all on the stream
        if (cudaMemcpyAsync(L_dev, L_host, lbytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(D_dev, D_host, dbytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SELINV_ERR_CUDA;
        const int rc = selinv_numeric(plan, dtype, L_dev, D_dev, Ainv_dev, stream);
        if (rc) return rc;
        return cudaMemcpyAsync(Ainv_host, Ainv_dev, lbytes, cudaMemcpyDeviceToHost, st) == cudaSuccess
                   ? SELINV_OK : SELINV_ERR_CUDA;
    };
    if ((p.opts.autotune && !p.tuned[dtype]) || (p.opts.debug_checks & 1) || p.opts.schedule != SELINV_SCHED_LEVEL)
        return whole();
    int rc = numeric_prepare(plan, dtype, L_dev, D_dev, Ainv_dev, st);
    if (rc) return rc;
    Schedule &S = plan->single;
    if (S.join_at < 0 || S.join_at >= (int)S.launches.size()) return whole();
    HostPipe &h = plan->host;
    if (host_pipe_init(h) != cudaSuccess) return SELINV_ERR_CUDA;
    const int ltop = S.launches[S.join_at].level;
    const int lmid = S.join_at2 >= 0 && S.join_at2 < (int)S.launches.size() ? S.launches[S.join_at2].level : p.nlevels;
    // runs of consecutive supernodes whose level is in [lo, hi), as byte ranges of the panels
    auto runs = [&](int lo, int hi) {
        std::vector<std::pair<size_t, size_t>> r;
        for (int32_t K = 0; K < p.ns;) {
            if (p.level[K] < lo || p.level[K] >= hi) { K++; continue; }
            int32_t K1 = K;
            while (K1 + 1 < p.ns && p.level[K1 + 1] >= lo && p.level[K1 + 1] < hi) K1++;
            r.push_back({es * (size_t)p.panel_off[K], es * (size_t)(p.panel_off[K1 + 1] - p.panel_off[K])});
            K = K1 + 1;
        }
        return r;
    };
    auto copies = [&](const std::vector<std::pair<size_t, size_t>> &r, const void *src, void *dst,
                      cudaMemcpyKind kind, cudaStream_t cst) -> cudaError_t {
        for (const auto &x : r) {
            const cudaError_t e = cudaMemcpyAsync(static_cast<char *>(dst) + x.first,
                                                  static_cast<const char *>(src) + x.first, x.second, kind, cst);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const int nl = p.nlevels;
    // D2H groups: [0, ltop), then level bounds at ~1/2 and ~4/5 of the rest's bytes
    std::vector<int> bounds{ltop};
    {
        std::vector<double> lb(nl, 0.0);
        for (int32_t K = 0; K < p.ns; K++) lb[p.level[K]] += (double)(p.panel_off[K + 1] - p.panel_off[K]);
        double rest = 0.0;
        for (int l = ltop; l < nl; l++) rest += lb[l];
        double acc = 0.0;
        size_t f = 0;
        const double frac[2] = {0.5, 0.8};
        for (int l = ltop; l < nl && f < 2; l++) {
            acc += lb[l];
            while (f < 2 && acc >= frac[f] * rest) {
                if (l + 1 < nl && l + 1 > bounds.back()) bounds.push_back(l + 1);
                f++;
            }
        }
    }
    IssueHooks hk;
    for (int b : bounds) {   // the first main launch of level b: all levels above it are done
        int at = (int)S.launches.size();
        for (int i = 0; i < (int)S.launches.size(); i++)
            if (!S.launches[i].side && S.launches[i].level >= b) { at = i; break; }
        hk.mark_at.push_back(at);
    }
    hk.mark_at.push_back((int)S.launches.size());   // the last group, after every launch
    std::vector<int> lo_of{0};
    for (int b : bounds) lo_of.push_back(b);
    cudaError_t e = cudaSuccess;
    hk.side_wait[0] = h.ev_mid;    // the side stream's phases wait for their panels of L
    hk.side_wait[1] = h.ev_rest;
    hk.mark = [&](int g) -> cudaError_t {
        const int lo = lo_of[g], hi = g < (int)bounds.size() ? bounds[g] : nl;
        cudaError_t x = cudaEventRecord(h.ev_grp[g], st);
        if (x == cudaSuccess) x = cudaStreamWaitEvent(h.cout, h.ev_grp[g], 0);
        if (x == cudaSuccess) x = copies(runs(lo, hi), Ainv_dev, Ainv_host, cudaMemcpyDeviceToHost, h.cout);
        return x;
    };
    auto body = [&]() -> cudaError_t {
        cudaError_t x;
        // inputs: everything that is on the stream before this call comes first
        if ((x = cudaEventRecord(h.ev_done, st)) != cudaSuccess ||
            (x = cudaStreamWaitEvent(h.cin, h.ev_done, 0)) != cudaSuccess ||
            (x = cudaStreamWaitEvent(h.cout, h.ev_done, 0)) != cudaSuccess ||
            (x = cudaMemcpyAsync(D_dev, D_host, dbytes, cudaMemcpyHostToDevice, h.cin)) != cudaSuccess ||
            (x = copies(runs(0, ltop), L_host, L_dev, cudaMemcpyHostToDevice, h.cin)) != cudaSuccess ||
            (x = cudaEventRecord(h.ev_top, h.cin)) != cudaSuccess ||
            (x = copies(runs(ltop, lmid), L_host, L_dev, cudaMemcpyHostToDevice, h.cin)) != cudaSuccess ||
            (x = cudaEventRecord(h.ev_mid, h.cin)) != cudaSuccess ||
            (x = copies(runs(lmid, nl), L_host, L_dev, cudaMemcpyHostToDevice, h.cin)) != cudaSuccess ||
            (x = cudaEventRecord(h.ev_rest, h.cin)) != cudaSuccess ||
            (x = cudaStreamWaitEvent(st, h.ev_top, 0)) != cudaSuccess)
            return x;
        if ((x = issue(S, st, false, &hk)) != cudaSuccess) return x;
        // the stream's completion covers both copy streams
        if ((x = cudaEventRecord(h.ev_in_done, h.cin)) != cudaSuccess ||
            (x = cudaStreamWaitEvent(st, h.ev_in_done, 0)) != cudaSuccess ||
            (x = cudaEventRecord(h.ev_done, h.cout)) != cudaSuccess)
            return x;
        return cudaStreamWaitEvent(st, h.ev_done, 0);
    };
    plan->last_stream = st;
    note_launch((int)S.launches.size());
    // with pinned host buffers the whole call (copies, kernels, the streams'
    // forks and joins) is captured once per set of buffers and replayed
    auto pinned = [](const void *q) {
        cudaPointerAttributes a;
        const bool ok = cudaPointerGetAttributes(&a, q) == cudaSuccess && a.type == cudaMemoryTypeHost;
        cudaGetLastError();
        return ok;
    };
    if (p.opts.use_graph && st != nullptr && st != cudaStreamLegacy && pinned(L_host) && pinned(D_host) &&
        pinned(Ainv_host)) {
        const std::array<const void *, 6> key{L_host, D_host, Ainv_host, L_dev, D_dev, Ainv_dev};
        if (!S.graph_host || S.host_key != key) {
            if (S.graph_host) cudaGraphExecDestroy(S.graph_host);
            S.graph_host = nullptr;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SELINV_ERR_CUDA;
            e = body();
            const cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (e != cudaSuccess || e2 != cudaSuccess || !g) {
                if (g) cudaGraphDestroy(g);
                return SELINV_ERR_CUDA;
            }
            if (programmatic_edges(g) != cudaSuccess) {
                cudaGraphDestroy(g);
                return SELINV_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&S.graph_host, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                S.graph_host = nullptr;
                return SELINV_ERR_CUDA;
            }
            S.host_key = key;
        }
        return cudaGraphLaunch(S.graph_host, st) == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
    }
    return body() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}

// The LU form (nonsymmetric values): the DFMA kernels with the descriptor's
// LU fields set; level schedule unless the plan asks for the plain one.
extern "C" int selinv_numeric_lu(selinv_plan plan, selinv_dtype dtype, const void *L, const void *Ut, void *Zl,
                                 void *Zu, void *stream) {
    NvtxRange nvtx_range("selinv_numeric_lu");
    if (!plan || (dtype != SELINV_F64 && dtype != SELINV_C128)) return SELINV_ERR_INVALID_ARG;
    PlanData &p = plan->data;
    if (p.ns == 0) return SELINV_OK;
    if (!L || !Ut || !Zl || !Zu || !aligned16(L) || !aligned16(Ut) || !aligned16(Zl) || !aligned16(Zu))
        return SELINV_ERR_INVALID_ARG;
    int rc = ensure_device(p);
    if (rc) return rc;
    if (plan->ws.empty()) plan->ws.resize(1);
    Workspace &w = plan->ws[0];
    if ((rc = w.ensure(p, dtype)) || (rc = w.ensure_lu(p))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Schedule &S = plan->lu;
    const int mode = p.opts.schedule == SELINV_SCHED_PLAIN ? SELINV_SCHED_PLAIN : SELINV_SCHED_LEVEL;
    if (!S.valid || S.key_L != L || S.key_D != Ut || S.key_Z != Zl || S.key_Z2 != Zu || S.key_dtype != dtype ||
        S.mode != mode) {
        ProbDesc d = make_desc(p, w, dtype, L, nullptr, Zl, false);
        d.lu = 1;
        d.symmetrize = 0;
        d.Ut = Ut;
        d.Zu = Zu;
        d.LDu = w.LDu;
        d.Vt = w.Vt;
        std::vector<const PlanData *> plans{&p};
        std::vector<ProbDesc> descs{d};
        rc = build_schedule(S, plans, descs, mode);
        if (rc) { S.valid = false; return rc; }
        S.spin_limit = p.opts.spin_limit;
        S.valid = true;
        S.key_L = L; S.key_D = Ut; S.key_Z = Zl; S.key_Z2 = Zu; S.key_dtype = dtype; S.mode = mode;
    }
    plan->last_stream = st;
    return run_schedule(S, st, p.opts.use_graph != 0);
}

extern "C" int selinv_numeric_profile(selinv_plan plan, selinv_dtype dtype, const void *L,
                                      const void *D, void *Z, void *stream, double *kernel_ms,
                                      int64_t *kernel_launches) {
    NvtxRange nvtx_range("selinv_numeric_profile");
    if (!kernel_ms || !kernel_launches) return SELINV_ERR_INVALID_ARG;
    // build (or reuse) the schedule through the normal path, without a graph
    if (!plan) return SELINV_ERR_INVALID_ARG;
    const int saved_graph = plan->data.opts.use_graph;
    plan->data.opts.use_graph = 0;
    int rc = selinv_numeric(plan, dtype, L, D, Z, stream);   // may autotune first
    plan->data.opts.use_graph = saved_graph;
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return SELINV_ERR_CUDA;
    Schedule &S = plan->single;
    std::vector<cudaEvent_t> ev(2 * S.launches.size());
    for (auto &e : ev) cudaEventCreate(&e);
    static_assert(KL_NKINDS == SELINV_PROFILE_KINDS, "profile kinds");
    for (int k = 0; k < KL_NKINDS; k++) { kernel_ms[k] = 0; kernel_launches[k] = 0; }
    if (issue_pre(S, st) != cudaSuccess) rc = SELINV_ERR_CUDA;
    for (size_t i = 0; i < S.launches.size(); i++) {
        const Launch &L = S.launches[i];
        cudaEventRecord(ev[2 * i], st);
        cudaError_t e = launch_one(S, L, st);
        cudaEventRecord(ev[2 * i + 1], st);
        if (e != cudaSuccess) rc = SELINV_ERR_CUDA;
    }
    note_launch((int)S.launches.size());
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = SELINV_ERR_CUDA;
    for (size_t i = 0; i < S.launches.size() && rc == SELINV_OK; i++) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
        kernel_ms[S.launches[i].kind] += ms;
        kernel_launches[S.launches[i].kind] += 1;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

extern "C" int selinv_numeric_batched(int nitems, const selinv_plan *plans, const selinv_dtype *dtypes,
                                      const void *const *L, const void *const *D, void *const *Z,
                                      void *stream) {
    NvtxRange nvtx_range("selinv_numeric_batched");
    if (nitems <= 0 || !plans || !dtypes || !L || !D || !Z) return SELINV_ERR_INVALID_ARG;
    selinv_plan owner = plans[0];
    if (!owner) return SELINV_ERR_INVALID_ARG;
    for (int i = 0; i < nitems; i++) {
        if (!plans[i] || (dtypes[i] != SELINV_F64 && dtypes[i] != SELINV_C128 && dtypes[i] != SELINV_C128H))
            return SELINV_ERR_INVALID_ARG;
        if (!L[i] || !D[i] || !Z[i] || !aligned16(L[i]) || !aligned16(D[i]) || !aligned16(Z[i]))
            return SELINV_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int mode = owner->data.opts.schedule;
    // cached schedule for this exact batch?
    BatchEntry *hit = nullptr;
    for (auto &b : owner->batch_cache) {
        if ((int)b.plans.size() != nitems || b.mode != mode) continue;
        bool same = true;
        for (int i = 0; i < nitems && same; i++)
            same = b.plans[i] == plans[i] && b.dtypes[i] == dtypes[i] && b.L[i] == L[i] &&
                   b.D[i] == D[i] && b.Z[i] == Z[i] && b.sel_version[i] == plans[i]->data.sel_version;
        if (same) { hit = &b; break; }
    }
    for (int i = 0; i < nitems; i++) {
        int rc = ensure_device(plans[i]->data);
        if (rc) return rc;
    }
    if (!hit) {
        // one workspace per batch item, owned by the first plan
        if ((int)owner->ws.size() < nitems + 1) owner->ws.resize(nitems + 1);
        std::vector<const PlanData *> pds(nitems);
        std::vector<ProbDesc> descs(nitems);
        for (int i = 0; i < nitems; i++) {
            int rc = owner->ws[i + 1].ensure(plans[i]->data, dtypes[i]);
            if (!rc && mode == SELINV_SCHED_PERSISTENT) rc = owner->ws[i + 1].ensure_persistent(plans[i]->data);
            if (rc) return rc;
            pds[i] = &plans[i]->data;
            descs[i] = make_desc(plans[i]->data, owner->ws[i + 1], dtypes[i], L[i], D[i], Z[i],
                                 mode == SELINV_SCHED_PERSISTENT);
            descs[i].status = owner->data.d_status;
        }
        if (owner->batch_cache.size() >= 4) {
            owner->batch_cache.front().sched.release();
            owner->batch_cache.erase(owner->batch_cache.begin());
        }
        owner->batch_cache.emplace_back();
        BatchEntry &b = owner->batch_cache.back();
        b.mode = mode;
        b.plans.assign(plans, plans + nitems);
        b.dtypes.assign(dtypes, dtypes + nitems);
        b.L.assign(L, L + nitems);
        b.D.assign(D, D + nitems);
        b.Z.assign(Z, Z + nitems);
        for (int i = 0; i < nitems; i++) b.sel_version.push_back(plans[i]->data.sel_version);
        int rc = build_schedule(b.sched, pds, descs, mode);
        if (rc) {
            b.sched.release();
            owner->batch_cache.pop_back();
            return rc;
        }
        b.sched.spin_limit = owner->data.opts.spin_limit;
        if (mode == SELINV_SCHED_PERSISTENT) {
            // both element types share one ticket: the launches run one after the other
            b.sched.ticket = owner->ws[1].ticket;
            b.sched.wait_on_unset = (owner->data.opts.debug_checks & 2) ? 1 : 0;
            for (int i = 0; i < nitems; i++) {
                b.sched.reset_ptr.push_back(owner->ws[i + 1].done);
                b.sched.reset_bytes.push_back(sizeof(int) * (size_t)(plans[i]->data.ns + 1));
            }
            b.sched.reset_ptr.push_back(owner->ws[1].ticket);
            b.sched.reset_bytes.push_back(sizeof(int));
        }
        hit = &b;
    }
    owner->last_stream = st;
    if (owner->data.opts.debug_checks & 1) {
        for (int i = 0; i < nitems; i++) {
            const int64_t w = dtypes[i] == SELINV_F64 ? 1 : 2;
            if (launch_check_finite(L[i], w * plans[i]->data.nnz, owner->data.d_status, st) != cudaSuccess ||
                launch_check_finite(D[i], w * plans[i]->data.n, owner->data.d_status, st) != cudaSuccess)
                return SELINV_ERR_CUDA;
            note_launch(2);
        }
    }
    return run_schedule(hit->sched, st, owner->data.opts.use_graph != 0);
}

extern "C" int selinv_status(selinv_plan plan) {
    if (!plan) return SELINV_ERR_INVALID_ARG;
    if (!plan->data.d_status) return SELINV_OK;
    if (cudaStreamSynchronize(plan->last_stream) != cudaSuccess) return SELINV_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, plan->data.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SELINV_ERR_CUDA;
    if (v) cudaMemset(plan->data.d_status, 0, sizeof(int));
    return v;
}

extern "C" const char *selinv_error_string(int code) {
    switch (code) {
    case SELINV_OK: return "ok";
    case SELINV_ERR_INVALID_ARG: return "invalid argument";
    case SELINV_ERR_BAD_ETREE: return "bad elimination tree (parent must be > child and own the first row below)";
    case SELINV_ERR_BAD_PATTERN: return "bad row pattern (rows must be sorted, start with the supernode's columns and be closed under the tree)";
    case SELINV_ERR_ZERO_PIVOT: return "zero pivot in D";
    case SELINV_ERR_NONFINITE: return "non-finite value in the input";
    case SELINV_ERR_OOM: return "out of memory";
    case SELINV_ERR_CUDA: return "CUDA error";
    case SELINV_ERR_TIMEOUT: return "a bounded device wait timed out";
    case SELINV_ERR_UNSUPPORTED: return "unsupported";
    case SELINV_ERR_BAD_INDEX: return "a gather address fell outside the panel array";
    default: return "unknown error";
    }
}

extern "C" int64_t selinv_launch_count(void) { return g_launches.load(); }
