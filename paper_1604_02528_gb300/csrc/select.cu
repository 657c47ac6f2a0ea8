// Subset selection and the pole-expansion sum.
//
// Only some entries of A^{-1} may be wanted (Sec. I: selected elements are
// all or a subset of the nonzero entries of the factors), e.g. the diagonal,
// or the entries of A's own pattern.  Alg. 1 computes supernode K from its
// ancestors' blocks only, so the supernodes that must run are the owners of
// the selected columns and all of their ancestors; every other subtree is
// left out of the schedules (build_schedule skips inactive supernodes).
//
// The pole-expansion sum is the consumer of a batch of selected inversions
// of shifted matrices A - z_l I sharing one pattern (density functional
// theory, the application Sec. I names first): out = sum_l w_l A_l^{-1}[pos],
// a fixed order of terms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "nvtx.h"
#include "plan.h"

namespace selinv {

template <typename T>
__global__ void k_gather_sel(const T *__restrict__ src, const int64_t *__restrict__ pos, int64_t n,
                             T *__restrict__ dst) {
    grid_dep_wait();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[pos[e]];
}

constexpr int kPoleChunk = 32;   // terms per launch (kernel parameters)
struct PoleTerms {
    const void *Z[kPoleChunk];
    double wr[kPoleChunk], wi[kPoleChunk];
    int cplx[kPoleChunk];
    int n;
    int accumulate;   // add to out (a later chunk of terms)
};

// out[e] (+)= sum_l w_l Z_l[pos[e]] in complex arithmetic, terms in order l
__global__ void k_pole_sum(const PoleTerms t, const int64_t *__restrict__ pos, int64_t n, double2 *__restrict__ out) {
    grid_dep_wait();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = pos[e];
        double2 acc = t.accumulate ? out[e] : make_double2(0.0, 0.0);
        for (int l = 0; l < t.n; l++) {
            double zr, zi;
            if (t.cplx[l]) {
                const double2 z = static_cast<const double2 *>(t.Z[l])[q];
                zr = z.x;
                zi = z.y;
            } else {
                zr = static_cast<const double *>(t.Z[l])[q];
                zi = 0.0;
            }
            acc.x = fma(t.wr[l], zr, fma(-t.wi[l], zi, acc.x));
            acc.y = fma(t.wr[l], zi, fma(t.wi[l], zr, acc.y));
        }
        out[e] = acc;
    }
}

static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace selinv

using namespace selinv;

extern "C" int selinv_plan_select(selinv_plan plan, int64_t nsel, const int32_t *rows, const int32_t *cols,
                                  int64_t *pos_out) {
    if (!plan || nsel < 0 || (nsel > 0 && (!rows || !cols))) return SELINV_ERR_INVALID_ARG;
    PlanData &p = plan->data;
    std::vector<uint8_t> active;
    std::vector<int64_t> pos;
    if (nsel > 0) {
        active.assign(std::max(p.ns, 1), 0);
        pos.resize(nsel);
        for (int64_t e = 0; e < nsel; e++) {
            int32_t r = rows[e], c = cols[e];
            if (r < 0 || c < 0 || r >= p.n || c >= p.n) return SELINV_ERR_INVALID_ARG;
            if (r < c) std::swap(r, c);   // symmetric: the stored lower entry
            // owner of column c, then row r in its row list (ascending)
            const int32_t K = (int32_t)(std::upper_bound(p.super_ptr.begin(), p.super_ptr.end(), c) -
                                        p.super_ptr.begin()) - 1;
            const int32_t *R0 = p.rows.data() + p.rowptr[K], *R1 = p.rows.data() + p.rowptr[K + 1];
            const int32_t *hit = std::lower_bound(R0, R1, r);
            if (hit == R1 || *hit != r) return SELINV_ERR_BAD_PATTERN;
            const int64_t ld = p.rowptr[K + 1] - p.rowptr[K];
            pos[e] = p.panel_off[K] + (int64_t)(c - p.super_ptr[K]) * ld + (hit - R0);
            // K and its ancestors run (stop at the first one already marked)
            for (int32_t J = K; J >= 0 && !active[J]; J = p.sparent[J]) active[J] = 1;
        }
    }
    if (pos_out && nsel > 0) std::memcpy(pos_out, pos.data(), sizeof(int64_t) * (size_t)nsel);
    p.active.swap(active);
    p.sel_pos.swap(pos);
    p.sel_version++;
    if (p.d_sel_pos) cudaFree(p.d_sel_pos);
    p.d_sel_pos = nullptr;
    // schedules built for the previous selection are stale
    plan->single.release();
    plan->single.valid = false;
    for (auto &b : plan->batch_cache) b.sched.release();
    plan->batch_cache.clear();
    return SELINV_OK;
}

extern "C" int64_t selinv_plan_selected(selinv_plan plan, int64_t *pos_out) {
    if (!plan) return SELINV_ERR_INVALID_ARG;
    const PlanData &p = plan->data;
    if (pos_out && !p.sel_pos.empty()) std::memcpy(pos_out, p.sel_pos.data(), sizeof(int64_t) * p.sel_pos.size());
    return (int64_t)p.sel_pos.size();
}

extern "C" int selinv_gather(selinv_plan plan, selinv_dtype dtype, const void *Ainv, void *out, void *stream) {
    NvtxRange nvtx_range("selinv_gather");
    if (!plan || (dtype != SELINV_F64 && dtype != SELINV_C128 && dtype != SELINV_C128H)) return SELINV_ERR_INVALID_ARG;
    PlanData &p = plan->data;
    const int64_t n = (int64_t)p.sel_pos.size();
    if (n == 0) return SELINV_OK;
    if (!Ainv || !out) return SELINV_ERR_INVALID_ARG;
    int rc = ensure_device(p);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!p.d_sel_pos) {
        if (cudaMalloc((void **)&p.d_sel_pos, sizeof(int64_t) * (size_t)n) != cudaSuccess) return SELINV_ERR_OOM;
        if (cudaMemcpy(p.d_sel_pos, p.sel_pos.data(), sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return SELINV_ERR_CUDA;
    }
    if (dtype == SELINV_F64)
        k_gather_sel<double><<<grid_for(n), 256, 0, st>>>(static_cast<const double *>(Ainv), p.d_sel_pos, n,
                                                          static_cast<double *>(out));
    else
        k_gather_sel<double2><<<grid_for(n), 256, 0, st>>>(static_cast<const double2 *>(Ainv), p.d_sel_pos, n,
                                                           static_cast<double2 *>(out));
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}

extern "C" int selinv_pole_sum(int nitems, const selinv_dtype *dtypes, const void *const *Ainv,
                               const double *weights, int64_t npos, const int64_t *pos, void *out, void *stream) {
    NvtxRange nvtx_range("selinv_pole_sum");
    if (nitems <= 0 || !dtypes || !Ainv || !weights || npos < 0) return SELINV_ERR_INVALID_ARG;
    if (npos == 0) return SELINV_OK;
    if (!pos || !out) return SELINV_ERR_INVALID_ARG;
    for (int l = 0; l < nitems; l++)
        if (!Ainv[l] || (dtypes[l] != SELINV_F64 && dtypes[l] != SELINV_C128 && dtypes[l] != SELINV_C128H))
            return SELINV_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int l0 = 0; l0 < nitems; l0 += kPoleChunk) {
        PoleTerms t;
        std::memset(&t, 0, sizeof(t));
        t.n = std::min(kPoleChunk, nitems - l0);
        t.accumulate = l0 > 0;
        for (int l = 0; l < t.n; l++) {
            t.Z[l] = Ainv[l0 + l];
            t.wr[l] = weights[2 * (l0 + l)];
            t.wi[l] = weights[2 * (l0 + l) + 1];
            t.cplx[l] = dtypes[l0 + l] != SELINV_F64;
        }
        k_pole_sum<<<grid_for(npos), 256, 0, st>>>(t, pos, npos, static_cast<double2 *>(out));
        note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}
