// Prerequisite factorization A = L D L^T without pivoting, supernodal,
// left-looking, level by level from the leaves (Sec. IV of the paper uses a
// supernodal factorization with a symmetric permutation and no dynamic
// pivoting; Sec. II-C: LDL^T for symmetric A).
//
//   k_assemble  scatter A's CSC values into the panels (after a memset)
//   k_fupdate   one row tile of supernode J pulls the updates of every
//               descendant K whose C meets J's columns:
//                 panel_J(rel(p), col(q)) -= sum_k L_K(p,k) D_K(k) L_K(q,k)
//               over the run of C_K owned by J (p >= q) -- the same owner
//               segments and relative indices the selected inversion
//               gathers with.  Each tile owns its rows: no atomics,
//               a fixed descendant order: deterministic.
//   k_fdiag     dense LDL^T of J's diagonal block in place (one CTA)
//   k_ftrsm     L(C,J) = A(C,J) L_JJ^{-T} D_J^{-1}, one thread per row
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "plan.h"
#include "seg_update.cuh"

namespace selinv {

constexpr int kFT = 64;  // rows per factor tile

template <typename T>
__global__ void k_assemble(const int64_t *__restrict__ pos, const T *__restrict__ vals, int64_t nnz,
                           T *__restrict__ L) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        L[pos[e]] = vals[e];
}

template <typename T>
__global__ void __launch_bounds__(256) k_fupdate(const FactorDesc *__restrict__ fd,
                                                 const int2 *__restrict__ tiles, int ntiles, int64_t tile0) {
    __shared__ SegSmem<T> sm;
    const int w = blockIdx.x;
    if (w >= ntiles) return;
    const FactorDesc &F = *fd;
    const int J = tiles[w].x;
    const int64_t ldJ = F.rowptr[J + 1] - F.rowptr[J];
    const int fcJ = F.super_ptr[J];
    T *PJ = static_cast<T *>(F.L) + F.panel_off[J];
    const T *Lall = static_cast<const T *>(F.L);
    const T *Dall = static_cast<const T *>(F.D);
    // (segment, p-range) pairs whose target rows fall in this tile, precomputed
    for (int64_t li = F.tseg_ptr[tile0 + w]; li < F.tseg_ptr[tile0 + w + 1]; li++) {
        const int4 ts = F.tseg[li];
        const int t = ts.x, pa = ts.y, np = ts.z - ts.y;
        const int K = F.seg_K[t];
        const int st = F.seg_start[t], nq = F.seg_end[t] - st;
        const int sK = F.super_ptr[K + 1] - F.super_ptr[K];
        const int64_t ldK = F.rowptr[K + 1] - F.rowptr[K];
        const int32_t *rel = F.relidx + F.rel_ptr[t];  // rel[p - st], p in [st, cK)
        const T *LC = Lall + F.panel_off[K] + sK;      // L_K(p, k) = LC[k*ldK + p]
        const T *DK = Dall + F.super_ptr[K];
        const int32_t *colq = F.rows + F.rowptr[K] + sK;
        __syncthreads();  // the previous segment's updates to this tile are complete
        auto x = [&](int pl, int k) { return mul(LC[(int64_t)k * ldK + pa + pl], DK[k]); };
        auto y = [&](int ql, int k) { return LC[(int64_t)k * ldK + st + ql]; };
        // the run's columns need not be consecutive columns of J: address by value
        auto out = [&](int pl, int ql, T u) {
            T *dst = PJ + (int64_t)(colq[st + ql] - fcJ) * ldJ + rel[pa + pl - st];
            *dst = sub(*dst, u);
        };
        seg_update<T>(pa, np, st, nq, sK, x, y, out, sm);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fdiag(const FactorDesc *__restrict__ fd,
                                               const int *__restrict__ js, int nj) {
    const int w = blockIdx.x;
    if (w >= nj) return;
    const FactorDesc &F = *fd;
    const int J = js[w];
    const int fc = F.super_ptr[J];
    const int s = F.super_ptr[J + 1] - fc;
    const int64_t ld = F.rowptr[J + 1] - F.rowptr[J];
    T *P = static_cast<T *>(F.L) + F.panel_off[J];
    T *D = static_cast<T *>(F.D) + fc;
    __shared__ T s_d;
    for (int j = 0; j < s; j++) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const T d = P[(int64_t)j * ld + j];
            if (is_zero(d) || !finite_val(d)) atomicCAS(F.status, 0, SELINV_ERR_ZERO_PIVOT);
            s_d = d;
            D[j] = d;
        }
        __syncthreads();
        const T rd = recip(s_d);
        for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) P[(int64_t)j * ld + i] = mul(P[(int64_t)j * ld + i], rd);
        __syncthreads();
        // a_ik -= L_ij d L_kj for j < k <= i < s
        const int m = s - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e % m, k = j + 1 + e / m;
            if (k > i) continue;
            T *a = P + (int64_t)k * ld + i;
            *a = sub(*a, mul(mul(P[(int64_t)j * ld + i], s_d), P[(int64_t)j * ld + k]));
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int i = e % s, k = e / s;
        if (i == k) P[(int64_t)k * ld + i] = Sc<T>::one();
        else if (i < k) P[(int64_t)k * ld + i] = Sc<T>::zero();
    }
}

template <typename T>
__global__ void __launch_bounds__(64) k_ftrsm(const FactorDesc *__restrict__ fd,
                                              const int2 *__restrict__ tiles, int ntiles) {
    const int w = blockIdx.x;
    if (w >= ntiles) return;
    const FactorDesc &F = *fd;
    const int J = tiles[w].x;
    const int fc = F.super_ptr[J];
    const int s = F.super_ptr[J + 1] - fc;
    const int64_t ld = F.rowptr[J + 1] - F.rowptr[J];
    const int64_t r = (int64_t)tiles[w].y * kFT + threadIdx.x;  // panel row
    if (r < s || r >= ld) return;
    T *P = static_cast<T *>(F.L) + F.panel_off[J];
    const T *D = static_cast<const T *>(F.D) + fc;
    // x (D L_JJ^T) = a : x_j = (a_j - sum_{k<j} x_k D_k L_jk) / D_j, in place
    for (int j = 0; j < s; j++) {
        T acc = P[(int64_t)j * ld + r];
        for (int k = 0; k < j; k++) msub(acc, mul(P[(int64_t)k * ld + r], D[k]), P[(int64_t)k * ld + j]);
        P[(int64_t)j * ld + r] = mul(acc, recip(D[j]));
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void factor_release(selinv_plan_s *plan) {
    FactorData *f = plan->factor;
    if (!f) return;
    auto fr = [](void *p) { if (p) cudaFree(p); };
    fr(f->d_a_pos); fr(f->d_seg_K); fr(f->d_seg_start); fr(f->d_seg_end); fr(f->d_seg_coloff);
    fr(f->d_dseg); fr(f->d_dseg_ptr); fr(f->d_rel_ptr); fr(f->d_tiles); fr(f->d_js); fr(f->d_desc);
    fr(f->d_tseg_ptr); fr(f->d_tseg);
    adjoint_release(f->adj);
    delete f;
    plan->factor = nullptr;
}

template <typename X>
static int up(X **d, const std::vector<X> &h) {
    *d = nullptr;
    if (cudaMalloc((void **)d, sizeof(X) * std::max<size_t>(1, h.size())) != cudaSuccess) return SELINV_ERR_OOM;
    if (!h.empty() && cudaMemcpy(*d, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SELINV_ERR_CUDA;
    return SELINV_OK;
}

// segment tables (descendant lists per owner) shared by factor and adjoint
int factor_tables(selinv_plan_s *plan) {
    FactorData *f = plan->factor;
    if (f->d_dseg) return SELINV_OK;
    const PlanData &p = plan->data;
    int rc = ensure_device(plan->data);
    if (rc) return rc;
    const size_t nseg = p.seg_owner.size();
    std::vector<int32_t> segK(nseg), segEnd(nseg);
    for (int32_t K = 0; K < p.ns; K++) {
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - (p.super_ptr[K + 1] - p.super_ptr[K]);
        for (int64_t t = p.seg_ptr[K]; t < p.seg_ptr[K + 1]; t++) {
            segK[t] = K;
            segEnd[t] = (t + 1 < p.seg_ptr[K + 1]) ? p.seg_start[t + 1] : (int32_t)c;
        }
    }
    std::vector<int64_t> dptr(p.ns + 1, 0);
    for (size_t t = 0; t < nseg; t++) dptr[p.seg_owner[t] + 1]++;
    for (int32_t J = 0; J < p.ns; J++) dptr[J + 1] += dptr[J];
    std::vector<int32_t> dseg(std::max<size_t>(1, nseg));
    {
        std::vector<int64_t> fl(dptr.begin(), dptr.end() - 1);
        for (size_t t = 0; t < nseg; t++) dseg[fl[p.seg_owner[t]]++] = (int32_t)t;  // ascending K
    }
    // per-level launch lists, leaves first
    f->h_tiles.clear(); f->h_js.clear();
    f->tile_lptr.assign(1, 0); f->j_lptr.assign(1, 0);
    for (int l = p.nlevels - 1; l >= 0; l--) {
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t J = p.level_list[e];
            const int64_t ld = p.rowptr[J + 1] - p.rowptr[J];
            for (int64_t t = 0; t < (ld + kFT - 1) / kFT; t++) f->h_tiles.push_back(make_int2(J, (int)t));
            f->h_js.push_back(J);
        }
        f->tile_lptr.push_back((int64_t)f->h_tiles.size());
        f->j_lptr.push_back((int64_t)f->h_js.size());
    }
    // per panel tile (launch order): the (segment, p-range) pairs that land in
    // it, in ascending segment order (the fixed summation order)
    {
        std::vector<int64_t> tile_of(p.ns + 1, 0);      // index of (J, tile 0) in h_tiles
        for (size_t w = 0; w < f->h_tiles.size(); w++)
            if (f->h_tiles[w].y == 0) tile_of[f->h_tiles[w].x] = (int64_t)w;
        std::vector<std::vector<int4>> lists(f->h_tiles.size());
        for (int32_t J = 0; J < p.ns; J++)
            for (int64_t di = dptr[J]; di < dptr[J + 1]; di++) {
                const int32_t t = dseg[di];
                const int32_t K = segK[t];
                const int64_t cK = p.rowptr[K + 1] - p.rowptr[K] - (p.super_ptr[K + 1] - p.super_ptr[K]);
                const int32_t *rel = p.relidx.data() + p.rel_ptr[t];
                int64_t q = p.seg_start[t];
                while (q < cK) {
                    const int32_t tl = rel[q - p.seg_start[t]] / kFT;
                    int64_t qe = q;
                    while (qe < cK && rel[qe - p.seg_start[t]] / kFT == tl) qe++;
                    lists[tile_of[J] + tl].push_back(make_int4(t, (int)q, (int)qe, 0));
                    q = qe;
                }
            }
        std::vector<int64_t> tptr(f->h_tiles.size() + 1, 0);
        std::vector<int4> tseg;
        for (size_t w = 0; w < lists.size(); w++) {
            tseg.insert(tseg.end(), lists[w].begin(), lists[w].end());
            tptr[w + 1] = (int64_t)tseg.size();
        }
        if ((rc = up(&f->d_tseg_ptr, tptr))) return rc;
        if ((rc = up(&f->d_tseg, tseg))) return rc;
    }
    if ((rc = up(&f->d_seg_K, segK))) return rc;
    if ((rc = up(&f->d_seg_start, p.seg_start))) return rc;
    if ((rc = up(&f->d_seg_end, segEnd))) return rc;
    if ((rc = up(&f->d_seg_coloff, p.seg_coloff))) return rc;
    if ((rc = up(&f->d_dseg_ptr, dptr))) return rc;
    if ((rc = up(&f->d_dseg, dseg))) return rc;
    if ((rc = up(&f->d_rel_ptr, p.rel_ptr))) return rc;
    if ((rc = up(&f->d_tiles, f->h_tiles))) return rc;
    if ((rc = up(&f->d_js, f->h_js))) return rc;
    if (cudaMalloc((void **)&f->d_desc, sizeof(FactorDesc)) != cudaSuccess) return SELINV_ERR_OOM;
    return SELINV_OK;
}

FactorDesc *factor_desc(selinv_plan_s *plan, void *L, void *D, cudaStream_t st) {
    FactorData *f = plan->factor;
    const PlanData &p = plan->data;
    FactorDesc h;
    h.super_ptr = p.d_super_ptr;
    h.rowptr = p.d_rowptr;
    h.rows = p.d_rows;
    h.panel_off = p.d_panel_off;
    h.relidx = p.d_relidx;
    h.rel_ptr = f->d_rel_ptr;
    h.seg_K = f->d_seg_K;
    h.seg_start = f->d_seg_start;
    h.seg_end = f->d_seg_end;
    h.seg_coloff = f->d_seg_coloff;
    h.dseg_ptr = f->d_dseg_ptr;
    h.dseg = f->d_dseg;
    h.tseg_ptr = f->d_tseg_ptr;
    h.tseg = f->d_tseg;
    h.L = L;
    h.D = D;
    h.status = p.d_status;
    cudaMemcpyAsync(f->d_desc, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    return f->d_desc;
}

template <typename T>
static int factor_t(selinv_plan_s *plan, const void *A, void *L, void *D, cudaStream_t st) {
    FactorData *f = plan->factor;
    const PlanData &p = plan->data;
    FactorDesc *fd = factor_desc(plan, L, D, st);
    if (cudaMemsetAsync(L, 0, sizeof(T) * (size_t)p.nnz, st) != cudaSuccess) return SELINV_ERR_CUDA;
    if (f->nnzA > 0) {
        const int blocks = (int)std::min<int64_t>((f->nnzA + 255) / 256, 152 * 8);
        k_assemble<T><<<blocks, 256, 0, st>>>(f->d_a_pos, static_cast<const T *>(A), f->nnzA, static_cast<T *>(L));
        note_launch();
    }
    const int nl = (int)f->tile_lptr.size() - 1;
    for (int l = 0; l < nl; l++) {
        const int64_t t0 = f->tile_lptr[l], t1 = f->tile_lptr[l + 1];
        const int64_t j0 = f->j_lptr[l], j1 = f->j_lptr[l + 1];
        if (t1 > t0) k_fupdate<T><<<(int)(t1 - t0), 256, 0, st>>>(fd, f->d_tiles + t0, (int)(t1 - t0), t0);
        if (j1 > j0) k_fdiag<T><<<(int)(j1 - j0), 256, 0, st>>>(fd, f->d_js + j0, (int)(j1 - j0));
        if (t1 > t0) k_ftrsm<T><<<(int)(t1 - t0), kFT, 0, st>>>(fd, f->d_tiles + t0, (int)(t1 - t0));
        note_launch(3);
    }
    return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}

}  // namespace selinv

using namespace selinv;

extern "C" int selinv_plan_set_matrix(selinv_plan plan, int32_t n, const int64_t *colptr,
                                      const int32_t *rowind) {
    if (!plan || !colptr || (n > 0 && !rowind) || n != plan->data.n) return SELINV_ERR_INVALID_ARG;
    const PlanData &p = plan->data;
    std::vector<int32_t> col2s(n);
    for (int32_t K = 0; K < p.ns; K++)
        for (int32_t j = p.super_ptr[K]; j < p.super_ptr[K + 1]; j++) col2s[j] = K;
    std::vector<int64_t> pos(colptr[n] > 0 ? colptr[n] : 0);
    for (int32_t j = 0; j < n; j++) {
        const int32_t K = col2s[j];
        const int32_t *R = p.rows.data() + p.rowptr[K];
        const int64_t m = p.rowptr[K + 1] - p.rowptr[K];
        int64_t t = j - p.super_ptr[K];
        for (int64_t e = colptr[j]; e < colptr[j + 1]; e++) {
            const int32_t i = rowind[e];
            if (i < j || i >= n) return SELINV_ERR_BAD_PATTERN;
            while (t < m && R[t] < i) t++;
            if (t >= m || R[t] != i) return SELINV_ERR_BAD_PATTERN;  // A not inside L's pattern
            pos[e] = p.panel_off[K] + (int64_t)(j - p.super_ptr[K]) * m + t;
        }
    }
    if (!plan->factor) plan->factor = new FactorData();
    FactorData *f = plan->factor;
    if (f->d_a_pos) cudaFree(f->d_a_pos);
    f->d_a_pos = nullptr;
    f->n = n;
    f->nnzA = (int64_t)pos.size();
    f->a_pos = pos;
    int rc = ensure_device(plan->data);
    if (rc) return rc;
    return up(&f->d_a_pos, f->a_pos);
}

extern "C" int selinv_factor(selinv_plan plan, selinv_dtype dtype, const void *A, void *L, void *D,
                             void *stream) {
    if (!plan || !plan->factor || (dtype != SELINV_F64 && dtype != SELINV_C128)) return SELINV_ERR_INVALID_ARG;
    if (plan->data.ns == 0) return SELINV_OK;
    if (!L || !D || (plan->factor->nnzA > 0 && !A)) return SELINV_ERR_INVALID_ARG;
    int rc = factor_tables(plan);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    plan->last_stream = st;
    return dtype == SELINV_C128 ? factor_t<zd>(plan, A, L, D, st) : factor_t<double>(plan, A, L, D, st);
}
