// Prerequisite factorization A = L D L^T without pivoting, supernodal, level
// by level from the leaves (Sec. IV of the paper uses a supernodal
// factorization with a symmetric permutation and no dynamic pivoting; Sec.
// II-C: LDL^T for symmetric A, L D L^H for a Hermitian one, where every
// transposed factor below is conjugated), in multifrontal form:
//
//   k_assemble  scatter A's CSC values into the panels (after a memset)
//   k_fasm      extend-add of each child's update matrix U_child into its
//               parent J: entries whose column is one of J's columns go to
//               J's panel, the rest into U_J (one launch per child rank, so
//               no two writers meet; fixed order: deterministic)
//   k_fdiag     dense LDL^T of J's diagonal block in place (one CTA)
//   k_ftrsm     L(C,J) = A(C,J) L_JJ^{-T} D_J^{-1}, one thread per row
//   k_fupd      U_J -= L_CJ D_J L_CJ^T (lower c x c, 64 x 64 tiles)
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "nvtx.h"
#include "plan.h"
#include "seg_update.cuh"

namespace selinv {

constexpr int kFT = 64;  // rows per factor tile

template <typename T>
__global__ void k_assemble(const int64_t *__restrict__ pos, const T *__restrict__ vals, int64_t nnz,
                           T *__restrict__ L) {
    grid_dep_wait();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        L[pos[e]] = vals[e];
}

// Extend-add of one child's update matrix into its parent J: entry (a, b),
// a >= b, of U_child lands at rows(J) positions (pa, pb) -- in J's panel when
// the column C_child[b] is one of J's columns, else in U_J.  One launch per
// child rank: two children of one parent never run together.
template <typename T>
__global__ void __launch_bounds__(256) k_fasm(const FactorDesc *__restrict__ fd, const int2 *__restrict__ items,
                                              int nitems) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const FactorDesc &F = *fd;
    const int ch = items[w].x, chunk = items[w].y;
    const int J = F.sparent[ch];
    const int sch = F.super_ptr[ch + 1] - F.super_ptr[ch];
    const int cch = (int)(F.rowptr[ch + 1] - F.rowptr[ch] - sch);
    const int sJ = F.super_ptr[J + 1] - F.super_ptr[J];
    const int64_t ldJ = F.rowptr[J + 1] - F.rowptr[J];
    const int cJ = (int)(ldJ - sJ);
    const int32_t *pos = F.chpos + F.rowptr[ch] + sch;
    const T *Uc = static_cast<const T *>(F.U) + F.u_off[ch];
    T *UJ = static_cast<T *>(F.U) + F.u_off[J];
    T *PJ = static_cast<T *>(F.L) + F.panel_off[J];
    const int64_t cc = (int64_t)cch * cch;
    for (int64_t e = (int64_t)chunk * kAsmChunk + threadIdx.x; e < cc && e < (int64_t)(chunk + 1) * kAsmChunk; e += 256) {
        const int a = (int)(e % cch), b = (int)(e / cch);
        if (a < b) continue;
        const T v = Uc[e];
        const int pa = pos[a], pb = pos[b];
        T *dst = pb < sJ ? PJ + (int64_t)pb * ldJ + pa : UJ + (int64_t)(pb - sJ) * cJ + (pa - sJ);
        *dst = add(*dst, v);
    }
}

// U_J -= L_CJ D_J L_CJ^T on one 64 x 64 tile of the lower c x c triangle
template <typename T>
__global__ void __launch_bounds__(256) k_fupd(const FactorDesc *__restrict__ fd, const int4 *__restrict__ items,
                                              int nitems) {
    grid_dep_wait();
    __shared__ SegSmem<T> sm;
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const FactorDesc &F = *fd;
    const int J = items[w].x, ti = items[w].y, tj = items[w].z;
    const int sJ = F.super_ptr[J + 1] - F.super_ptr[J];
    const int64_t ld = F.rowptr[J + 1] - F.rowptr[J];
    const int c = (int)(ld - sJ);
    const T *LC = static_cast<const T *>(F.L) + F.panel_off[J] + sJ;   // L(p, k) = LC[k*ld + p]
    const T *DJ = static_cast<const T *>(F.D) + F.super_ptr[J];
    T *UJ = static_cast<T *>(F.U) + F.u_off[J];
    const int pa = ti * kSegB, st = tj * kSegB;
    const int np = c - pa < kSegB ? c - pa : kSegB, nq = c - st < kSegB ? c - st : kSegB;
    auto x = [&](int pl, int k) { return mul(LC[(int64_t)k * ld + pa + pl], DJ[k]); };
    auto y = [&](int ql, int k) { return cjif(LC[(int64_t)k * ld + st + ql], F.herm != 0); };
    auto out = [&](int pl, int ql, T v) {
        T *dst = UJ + (int64_t)(st + ql) * c + pa + pl;
        *dst = sub(*dst, v);
    };
    seg_update<T>(pa, np, st, nq, sJ, x, y, out, sm);
}

template <typename T>
__global__ void __launch_bounds__(256) k_fdiag(const FactorDesc *__restrict__ fd,
                                               const int *__restrict__ js, int nj) {
    grid_dep_wait();
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
            *a = sub(*a, mul(mul(P[(int64_t)j * ld + i], s_d), cjif(P[(int64_t)j * ld + k], F.herm != 0)));
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
    grid_dep_wait();
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
    // x (D L_JJ^T) = a : x_j = (a_j - sum_{k<j} x_k D_k L_jk) / D_j, in place (conj(L_jk): Hermitian)
    const bool h = F.herm != 0;
    for (int j = 0; j < s; j++) {
        T acc = P[(int64_t)j * ld + r];
        for (int k = 0; k < j; k++) msub(acc, mul(P[(int64_t)k * ld + r], D[k]), cjif(P[(int64_t)k * ld + j], h));
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
    fr(f->d_a_pos); fr(f->d_tiles); fr(f->d_js); fr(f->d_desc);
    fr(f->d_asm); fr(f->d_uitems); fr(f->d_uoff); fr(f->d_chpos); fr(f->U);
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

// launch lists and update-matrix tables, shared by the factorization and
// the selected-inversion adjoint
int factor_tables(selinv_plan_s *plan) {
    FactorData *f = plan->factor;
    if (f->d_desc) return SELINV_OK;
    const PlanData &p = plan->data;
    int rc = ensure_device(plan->data);
    if (rc) return rc;
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
    // update matrices: offsets; the position of every C_K entry in its
    // parent's row list (closure: C_K lies inside rows(parent)); children by rank
    f->u_off.assign(p.ns + 1, 0);
    for (int32_t K = 0; K < p.ns; K++) {
        const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - (p.super_ptr[K + 1] - p.super_ptr[K]);
        f->u_off[K + 1] = f->u_off[K] + c * c;
    }
    f->chpos.assign(std::max<int64_t>(p.rowptr[p.ns], 1), 0);
    std::vector<int> rank(p.ns, 0), nchild(p.ns, 0);
    for (int32_t K = 0; K < p.ns; K++) {
        const int32_t P = p.sparent[K];
        if (P < 0) continue;
        rank[K] = nchild[P]++;
        const int s = p.super_ptr[K + 1] - p.super_ptr[K];
        const int32_t *RP = p.rows.data() + p.rowptr[P];
        const int64_t mP = p.rowptr[P + 1] - p.rowptr[P];
        int64_t t = 0;
        for (int64_t r = p.rowptr[K] + s; r < p.rowptr[K + 1]; r++) {   // both lists ascending
            while (t < mP && RP[t] < p.rows[r]) t++;
            f->chpos[r] = (int32_t)t;
        }
    }
    f->npass = 1;
    for (int32_t K = 0; K < p.ns; K++) f->npass = std::max(f->npass, nchild[K]);
    std::vector<int64_t> kid_ptr(p.ns + 1, 0);
    for (int32_t K = 0; K < p.ns; K++) kid_ptr[K + 1] = kid_ptr[K] + nchild[K];
    std::vector<int32_t> kids(std::max<int64_t>(kid_ptr[p.ns], 1));
    for (int32_t K = 0; K < p.ns; K++)
        if (p.sparent[K] >= 0) kids[kid_ptr[p.sparent[K]] + rank[K]] = K;
    f->asm_items.clear(); f->uitems.clear();
    f->asm_lptr.assign(1, 0);
    f->u_lptr.assign(1, 0);
    for (int l = p.nlevels - 1; l >= 0; l--) {
        for (int r = 0; r < f->npass; r++) {
            for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                const int32_t K = p.level_list[e];
                if (r >= nchild[K]) continue;
                const int32_t ch = kids[kid_ptr[K] + r];
                const int64_t cc = f->u_off[ch + 1] - f->u_off[ch];
                for (int64_t ck = 0; ck < (cc + kAsmChunk - 1) / kAsmChunk; ck++) f->asm_items.push_back(make_int2(ch, (int)ck));
            }
            f->asm_lptr.push_back((int64_t)f->asm_items.size());
        }
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t K = p.level_list[e];
            const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - (p.super_ptr[K + 1] - p.super_ptr[K]);
            const int nt = (int)((c + kSegB - 1) / kSegB);
            for (int ti = 0; ti < nt; ti++)
                for (int tj = 0; tj <= ti; tj++) f->uitems.push_back(make_int4(K, ti, tj, 0));
        }
        f->u_lptr.push_back((int64_t)f->uitems.size());
    }
    if ((rc = up(&f->d_tiles, f->h_tiles))) return rc;
    if ((rc = up(&f->d_js, f->h_js))) return rc;
    if ((rc = up(&f->d_asm, f->asm_items))) return rc;
    if ((rc = up(&f->d_uitems, f->uitems))) return rc;
    if ((rc = up(&f->d_uoff, f->u_off))) return rc;
    if ((rc = up(&f->d_chpos, f->chpos))) return rc;
    if (cudaMalloc((void **)&f->d_desc, sizeof(FactorDesc)) != cudaSuccess) return SELINV_ERR_OOM;
    return SELINV_OK;
}

FactorDesc *factor_desc(selinv_plan_s *plan, void *L, void *D, cudaStream_t st, int herm) {
    FactorData *f = plan->factor;
    const PlanData &p = plan->data;
    FactorDesc h;
    h.super_ptr = p.d_super_ptr;
    h.sparent = p.d_sparent;
    h.rowptr = p.d_rowptr;
    h.rows = p.d_rows;
    h.panel_off = p.d_panel_off;
    h.u_off = f->d_uoff;
    h.chpos = f->d_chpos;
    h.U = f->U;
    h.L = L;
    h.D = D;
    h.status = p.d_status;
    h.herm = herm;
    cudaMemcpyAsync(f->d_desc, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    return f->d_desc;
}

template <typename T>
static int factor_t(selinv_plan_s *plan, const void *A, void *L, void *D, cudaStream_t st, int herm) {
    FactorData *f = plan->factor;
    const PlanData &p = plan->data;
    const size_t ubytes = sizeof(T) * (size_t)std::max<int64_t>(f->u_off[p.ns], 1);
    if (f->U_bytes < ubytes) {
        if (f->U) cudaFree(f->U);
        f->U = nullptr;
        f->U_bytes = 0;
        if (cudaMalloc(&f->U, ubytes) != cudaSuccess) return SELINV_ERR_OOM;
        f->U_bytes = ubytes;
    }
    FactorDesc *fd = factor_desc(plan, L, D, st, herm);
    if (cudaMemsetAsync(L, 0, sizeof(T) * (size_t)p.nnz, st) != cudaSuccess) return SELINV_ERR_CUDA;
    if (cudaMemsetAsync(f->U, 0, ubytes, st) != cudaSuccess) return SELINV_ERR_CUDA;
    if (f->nnzA > 0) {
        const int blocks = (int)std::min<int64_t>((f->nnzA + 255) / 256, 152 * 8);
        k_assemble<T><<<blocks, 256, 0, st>>>(f->d_a_pos, static_cast<const T *>(A), f->nnzA, static_cast<T *>(L));
        note_launch();
    }
    const int nl = (int)f->tile_lptr.size() - 1;
    for (int l = 0; l < nl; l++) {
        // the children's update matrices complete J's panel and start U_J
        for (int r = 0; r < f->npass; r++) {
            const int64_t x0 = f->asm_lptr[l * f->npass + r], x1 = f->asm_lptr[l * f->npass + r + 1];
            if (x1 > x0) { k_fasm<T><<<(int)(x1 - x0), 256, 0, st>>>(fd, f->d_asm + x0, (int)(x1 - x0)); note_launch(); }
        }
        const int64_t t0 = f->tile_lptr[l], t1 = f->tile_lptr[l + 1];
        const int64_t j0 = f->j_lptr[l], j1 = f->j_lptr[l + 1];
        const int64_t u0 = f->u_lptr[l], u1 = f->u_lptr[l + 1];
        if (j1 > j0) k_fdiag<T><<<(int)(j1 - j0), 256, 0, st>>>(fd, f->d_js + j0, (int)(j1 - j0));
        if (t1 > t0) k_ftrsm<T><<<(int)(t1 - t0), kFT, 0, st>>>(fd, f->d_tiles + t0, (int)(t1 - t0));
        if (u1 > u0) k_fupd<T><<<(int)(u1 - u0), 256, 0, st>>>(fd, f->d_uitems + u0, (int)(u1 - u0));
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
    NvtxRange nvtx_range("selinv_factor");
    if (!plan || !plan->factor || (dtype != SELINV_F64 && dtype != SELINV_C128 && dtype != SELINV_C128H))
        return SELINV_ERR_INVALID_ARG;
    if (plan->data.ns == 0) return SELINV_OK;
    if (!L || !D || (plan->factor->nnzA > 0 && !A)) return SELINV_ERR_INVALID_ARG;
    int rc = factor_tables(plan);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    plan->last_stream = st;
    return dtype == SELINV_F64 ? factor_t<double>(plan, A, L, D, st, 0)
                               : factor_t<zd>(plan, A, L, D, st, dtype == SELINV_C128H);
}
