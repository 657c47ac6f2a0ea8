// Reverse mode of the selected inversion and of the LDL^T factorization
// (FP64).  The paper has no adjoint; this is the chain rule through the
// steps of Alg. 1 taken in reverse order.  Every accumulation has one owner
// and a fixed order (deterministic, no floating-point atomics).
//
// Selected-inversion adjoint, leaves -> root.  With Zbar the cotangent of
// every stored lower entry of A^{-1}, for each K:
//   Zbar on K's panel is completed by the extend-add of its children's
//   update matrices V (below), which also starts V_K            [k_adj_asm]
//   S      = symmetric cotangent of the diagonal block (S_ii = Zbar_ii,
//            S_ij = S_ji = Zbar_ij / 2)                       [k_adj_ybar]
//   Ybar   = Zbar_{C,K} - Lhat S                              [k_adj_ybar]
//   V_K   -= sym(Ybar Lhat^T): the cotangent that the gather of A^{-1}(C,C)
//            sends to the ancestors, handed to the parent as a dense c x c
//            update matrix (multifrontal style: entries whose column belongs
//            to the parent go to its panel, the rest into its own V)  [k_adj_vupd]
//   Lhatb  = -Y S - A^{-1}_{C,C} Ybar  (the gather recomputed) [k_adj_lhbar]
//   Lbar_CK = Lhatb M^T, M = L_KK^{-1}; Mbar = L_CK^T Lhatb + 2 D^{-1} M S;
//   Lbar_KK = -(M^T Mbar M^T) strictly lower; Dbar_k = -(M S M^T)_kk / D_k^2
//                                            [k_adj_lhbar, k_adj_gemm, k_adj_sel_*]
// Factorization adjoint, root -> leaves (reverse of k_fupdate / k_fdiag / k_ftrsm):
//   Lbar_CJ -= (Abar(C,C) L_CJ) o D, the gathered Abar with its diagonal
//   doubled; Dbar_k -= 1/2 (L_CJ^T Abar(C,C) L_CJ)_kk          [k_fadj_pull]
//   Abar_CJ = Lbar_CJ D^{-1} L_JJ^{-1}; Nbar = A_CJ^T Lbar_CJ   [k_fadj_trsm]
//   Ubar = -N^T Nbar N^T with N = L_JJ^{-T} D^{-1}  [k_fadj_nbar, k_adj_gemm, k_fadj_ubar]
//   then the reverse of the dense LDL^T of the diagonal block in closed form
//                                                   [k_adj_gemm, k_fadj_fold]
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "nvtx.h"
#include "plan.h"
#include "fixedpoint.cuh"
#include "tile_gemm.cuh"
#include "seg_update.cuh"

namespace selinv {

constexpr int kNumSMs = 152;   // GB300
constexpr int kFinY = 4;   // CTAs per supernode (grid y) of the per-supernode s x s steps
constexpr int kAdjWideC = 256;   // rows of C from which any supernode takes the split (wide) path
constexpr int kRowSimtS = 32;    // levels whose wide supernodes are this narrow: row products on the FP64 kernel
// levels whose row products have fewer multiply-adds run them as 16 x 16 FP64
// tiles: measured at the top of the 24^3 tree, 1.8e6 of them take 11-14 us
// there against ~30 us (+ a digit pass) on tcgen05, 6e6 take 40-59 us
constexpr double kSmallProdFma = 2.5e6;

struct AdjDesc {
    const int32_t *super_ptr;
    const int64_t *rowptr;
    const int32_t *rows;
    const int64_t *panel_off;
    const int64_t *colbase, *relbase;
    const int32_t *relidx;
    const int64_t *linv_off, *part_off;
    const double *L, *D, *Z, *LD, *Linv;
    double *Zb;       // working cotangent of A^{-1} (panels)
    double *YB;       // S in the diagonal block, Ybar below (panels)
    double *Lb;       // Lbar (panels)
    double *Db;       // Dbar [n]
    double *Ab;       // Abar (panels)
    double *partial;  // split partials
    int *counter;     // per-supernode tile counters
    double *fin;      // per-supernode s x s scratch: 4 slots at 4*linv_off
    const int32_t *sparent;
    const int64_t *v_off;   // update matrix of K: c x c column-major at V + v_off[K]
    const int32_t *chpos;   // row-list position p of C_K[q]: its position in rows(parent(K))
    double *V;              // update matrices: the part of Zbar(C,C) not yet handed to an owner
    double *G;              // panels: -A^{-1}(C,C) Ybar, then Lhat_bar (supernodes on the split path)
};

struct AdjData {
    bool built = false;
    std::vector<Item> items;          // (J, tile, ntiles) per level, levels deepest first
    std::vector<int64_t> lvl_ptr;     // per level: [start, end) of items, buckets sorted
    std::vector<int> lvl_bucket_ptr;  // per level x bucket offsets (kNumBuckets+1 per level)
    std::vector<int2> linv_work;
    std::vector<Item> lhat_items;
    std::vector<int> lhat_bptr;
    std::vector<int2> gitems, citems;  // per level: (J, 16x16 tile) and (J, chunk | ntiles << 16)
    std::vector<int> js;               // per level: supernodes
    std::vector<int2> cz_work;         // per level: (J, 8-column block)
    std::vector<int64_t> cz_lptr;
    int2 *d_cz = nullptr;
    std::vector<int4> vitems;          // per level: (J, 32-row tile, 32-column tile) of the lower c x c
    std::vector<int64_t> v_lptr;
    int4 *d_vitems = nullptr;
    std::vector<int64_t> g_lptr, c_lptr, j_lptr;
    double *V = nullptr;  // update matrices (tables shared with the factorization)
    Item *d_items = nullptr, *d_lhat = nullptr;
    int2 *d_linv = nullptr, *d_gitems = nullptr, *d_citems = nullptr;
    int *d_js = nullptr;
    double *YB = nullptr, *Zb = nullptr, *Lbw = nullptr, *Ab = nullptr, *fin = nullptr;
    AdjDesc *d_desc = nullptr;
    ProbDesc *d_pdesc = nullptr;
    // Both adjoints, split by supernode width (rebuilt when the
    // options change).  Wide supernodes (s >= the tensor-core threshold) run
    // the gather-GEMM on the tcgen05 kernel and their c x s by s x s products
    // as (K, 32-row block, 32-column chunk) and (K, 64-row tile, chunk, 32-row block of s) items; narrow
    // ones keep the fused one-CTA-per-tile kernels.  Lists per level, deepest first.
    int split_key = -1;
    std::vector<Item> sm_items;               // narrow: (K, tile) per level x bucket
    std::vector<int> sm_bptr;
    std::vector<Item> wd_items;               // wide: (K, tile) per level
    std::vector<int64_t> wd_lptr;
    // row_items: (K, 32-row block, chunk, 0) of the row products of the wide
    // supernodes of levels whose widest is kRowSimtS columns or less (FP64
    // kernel; other levels: pr_items on tcgen05); mbp_items: (K, tile, chunk,
    // row block) of the split partials
    std::vector<int4> row_items, mbp_items;
    std::vector<int64_t> row_lptr, mbp_lptr;
    // rg_items: (K, 16 x 16 tile) of the row products on levels of fewer than
    // kSmallProdFma multiply-adds per product
    std::vector<int2> rg_items;
    std::vector<int64_t> rg_lptr;
    int2 *d_rg = nullptr;
    std::vector<int2> dig_work;               // wide with c > 0: (0, K << 8 | 8-column block)
    std::vector<int64_t> dig_lptr;
    std::vector<std::vector<int>> tc_launch;  // per level: tcgen05 and reduction launches of `tcs`
    Schedule tcs;                             // their items, split-k reductions and slab
    Schedule tcn;                             // the forward's normalization (L_KK^{-1}, Dinv, Lhat) of every supernode
    Item *d_sm = nullptr, *d_wd = nullptr;
    int4 *d_row = nullptr, *d_mbp = nullptr;
    int2 *d_dig = nullptr;
    ProbDesc *d_tcdesc = nullptr;
    int *cy = nullptr;                        // column maxima the tcgen05 launches record (unused here)
    // the per-level loops of the two passes as CUDA graphs (captured on first
    // use, rebuilt when the lists or the workspace change)
    int gen = 0;                              // bumped whenever the lists are rebuilt
    cudaGraphExec_t g_sel = nullptr, g_fac = nullptr;
    int g_sel_n = 0, g_fac_n = 0;             // launches in each graph
    long long g_sel_key = -1, g_fac_key = -1;
    const void *g_sel_ws = nullptr, *g_fac_ws = nullptr;
    // row products of the wide supernodes on the transposed tcgen05 kernel:
    // (K, 64-row tile) items and (K, 8-column block) digit work per level, the
    // digit planes of the s x s factor (7 x roundup(s, 64) x roundup(s, 16) per
    // supernode) and its column exponents, one descriptor per product
    std::vector<Item> pr_items;
    std::vector<int64_t> pr_lptr;
    std::vector<int2> sd_work;
    std::vector<int64_t> sd_lptr;
    Item *d_pr = nullptr;
    int2 *d_sdw = nullptr;
    uint16_t *sd = nullptr;
    int64_t *d_sd_off = nullptr;
    int *sdexp = nullptr;
    ProbDesc *d_pdp = nullptr;               // [5]: YBAR, LHB, LBC, FAC, FABAR
    // the update V_K -= sym(Ybar Lhat^T) of the wide supernodes on the
    // transposed tcgen05 kernel (SYRK mode): digit work (K, 32-row block) and
    // items (K, 128 x 64 tile) per level, the digit planes of [Ybar, Lhat]
    // (offsets restart at every level) and their row exponents; the narrow
    // supernodes keep k_adj_vupd (vn: their items)
    std::vector<int2> sy_work;
    std::vector<int64_t> sy_wlptr;
    std::vector<Item> sy_items;
    std::vector<int64_t> sy_lptr;
    std::vector<int4> vn_items;
    std::vector<int64_t> vn_lptr;
    int2 *d_syw = nullptr;
    Item *d_sy = nullptr;
    int4 *d_vn = nullptr;
    uint16_t *sy = nullptr;
    int64_t *d_sy_off = nullptr;
    int *syexp = nullptr;
    ProbDesc *d_sydesc = nullptr;
};

// ---------------------------------------------------------------------------
// Extend-add of one child's update matrix into its parent K (multifrontal
// hand-off): entry (a, b), a >= b, of V_child lands at rows(K) positions
// (pa, pb); into K's panel cotangent when C_child[b] is one of K's columns,
// else into V_K.  One launch per child rank, so two children of one parent
// never run together: no conflicts, a fixed order.
__global__ void __launch_bounds__(256) k_adj_asm(const AdjDesc *__restrict__ ad, const int2 *__restrict__ items,
                                                 int nitems) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const int ch = items[w].x, chunk = items[w].y;
    const int K = A.sparent[ch];
    const int sch = A.super_ptr[ch + 1] - A.super_ptr[ch];
    const int cch = (int)(A.rowptr[ch + 1] - A.rowptr[ch] - sch);
    const int sK = A.super_ptr[K + 1] - A.super_ptr[K];
    const int64_t ldK = A.rowptr[K + 1] - A.rowptr[K];
    const int cK = (int)(ldK - sK);
    const int32_t *pos = A.chpos + A.rowptr[ch] + sch;
    const double *Vc = A.V + A.v_off[ch];
    double *VK = A.V + A.v_off[K];
    double *ZbK = A.Zb + A.panel_off[K];
    const int64_t cc = (int64_t)cch * cch;
    for (int64_t e = (int64_t)chunk * kAsmChunk + threadIdx.x; e < cc && e < (int64_t)(chunk + 1) * kAsmChunk; e += 256) {
        const int a = (int)(e % cch), b = (int)(e / cch);
        if (a < b) continue;
        const double v = Vc[e];
        const int pa = pos[a], pb = pos[b];
        if (pb < sK) ZbK[(int64_t)pb * ldK + pa] += v;
        else VK[(int64_t)(pb - sK) * cK + (pa - sK)] += v;
    }
}

// V_K -= sym(Ybar Lhat^T) on one 32 x 32 tile of the lower c x c triangle
// (four times the CTAs of 64 x 64 tiles for the few supernodes of the top
// levels): [Ybar, Lhat] [Lhat, Ybar]^T over k' < 2s, the diagonal counted once
constexpr int kVB = 32;
__global__ void __launch_bounds__(256) k_adj_vupd(const AdjDesc *__restrict__ ad, const int4 *__restrict__ items,
                                                  int nitems) {
    grid_dep_wait();
    __shared__ SegSmem<double, kVB> sm;
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const int K = items[w].x, ti = items[w].y, tj = items[w].z;
    const int sK = A.super_ptr[K + 1] - A.super_ptr[K];
    const int64_t ld = A.rowptr[K + 1] - A.rowptr[K];
    const int c = (int)(ld - sK);
    const double *Yb = A.YB + A.panel_off[K] + sK;   // Ybar(p, k) = Yb[k*ld + p]
    const double *Lh = A.LD + A.panel_off[K] + sK;   // Lhat(p, k)
    double *VK = A.V + A.v_off[K];
    const int pa = ti * kVB, st = tj * kVB;
    const int np = c - pa < kVB ? c - pa : kVB, nq = c - st < kVB ? c - st : kVB;
    auto x = [&](int pl, int k) {
        return k < sK ? Yb[(int64_t)k * ld + pa + pl] : Lh[(int64_t)(k - sK) * ld + pa + pl];
    };
    auto y = [&](int ql, int k) {
        return k < sK ? Lh[(int64_t)k * ld + st + ql] : Yb[(int64_t)(k - sK) * ld + st + ql];
    };
    auto out = [&](int pl, int ql, double v) {
        if (pa + pl == st + ql) v *= 0.5;
        VK[(int64_t)(st + ql) * c + pa + pl] -= v;
    };
    seg_update<double, decltype(x), decltype(y), decltype(out), kVB>(pa, np, st, nq, 2 * sK, x, y, out, sm);
}

// The forward writes whole diagonal blocks (the strictly upper part holds
// copies of the lower entries), so a cotangent may arrive on an upper slot:
// add it to the lower mirror and clear it, one CTA per supernode.  Every
// later step reads only the lower triangle of a diagonal block.  Grid
// (supernodes, kFinY).
__global__ void __launch_bounds__(256) k_adj_fold(const AdjDesc *__restrict__ ad, int ns) {
    grid_dep_wait();
    const int K = blockIdx.x;
    if (K >= ns) return;
    const AdjDesc &A = *ad;
    const int s = A.super_ptr[K + 1] - A.super_ptr[K];
    const int64_t ld = A.rowptr[K + 1] - A.rowptr[K];
    double *Zb = A.Zb + A.panel_off[K];
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < s * s; e += gridDim.y * blockDim.x) {
        const int i = e % s, j = e / s;
        if (i <= j) continue;
        const double up = Zb[(int64_t)i * ld + j];
        if (up != 0.0) {
            Zb[(int64_t)j * ld + i] += up;
            Zb[(int64_t)i * ld + j] = 0.0;
        }
    }
}

// S (tile 0) and Ybar rows of one tile
__global__ void __launch_bounds__(256) k_adj_ybar(const AdjDesc *__restrict__ ad,
                                                  const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const Item it = items[w];
    const int J = it.K;
    const int s = A.super_ptr[J + 1] - A.super_ptr[J];
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const int c = (int)(ld - s);
    const double *Zb = A.Zb + A.panel_off[J];
    double *YB = A.YB + A.panel_off[J];
    const double *Lh = A.LD + A.panel_off[J] + s;
    auto S = [&](int a, int b) -> double {
        if (a == b) return Zb[(int64_t)b * ld + a];
        return 0.5 * (a > b ? Zb[(int64_t)b * ld + a] : Zb[(int64_t)a * ld + b]);
    };
    if (it.tile == 0)
        for (int e = threadIdx.x; e < s * s; e += blockDim.x) YB[(int64_t)(e / s) * ld + e % s] = S(e % s, e / s);
    const int p0 = it.tile * kTM;
    const int pm = c - p0 < kTM ? c - p0 : kTM;
    for (int e = threadIdx.x; e < pm * s; e += blockDim.x) {
        const int p = p0 + e % pm, j = e / pm;
        double v = Zb[(int64_t)j * ld + s + p];
        for (int k = 0; k < s; k++) v = fma(-Lh[(int64_t)k * ld + p], S(k, j), v);
        YB[(int64_t)j * ld + s + p] = v;
    }
}

// Lhat_bar rows of one tile (gather-GEMM with B = Ybar), the split Mbar term,
// then Lbar_C rows.
template <int TN>
__global__ void __launch_bounds__(kThreads) k_adj_lhbar(const AdjDesc *__restrict__ ad,
                                                        const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    using Sh = Shape<TN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *As = reinterpret_cast<double *>(smem_raw);
    double *Bs = As + kTK * (kTM > TN ? kTM : TN);
    double *Rows = Bs + kTK * TN;                         // [TM][TN] Lhat_bar rows of the tile
    __shared__ int64_t tile_cb[kTM], tile_rb[kTM];
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const Item it = items[w];
    const int J = it.K;
    const int s = A.super_ptr[J + 1] - A.super_ptr[J];
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const int c = (int)(ld - s);
    const int p0 = it.tile * kTM;
    const int pm = c - p0 < kTM ? c - p0 : kTM;
    const int64_t pos0 = A.rowptr[J] + s;
    const int64_t off = A.panel_off[J];
    for (int e = threadIdx.x; e < kTM; e += kThreads) {
        const int p = p0 + e;
        tile_cb[e] = p < c ? A.colbase[pos0 + p] : 0;
        tile_rb[e] = p < c ? A.relbase[pos0 + p] : 0;
    }
    double acc[Sh::MI][Sh::NJ];
#pragma unroll
    for (int i = 0; i < Sh::MI; i++)
#pragma unroll
        for (int j = 0; j < Sh::NJ; j++) acc[i][j] = 0.0;
    if (pm > 0) {
        LoadGather<double, TN> la{A.Z, A.colbase + pos0, A.relbase + pos0, A.relidx, tile_cb, tile_rb, p0, c};
        LoadColMajor<double, TN> lb{A.YB + off + s, ld, c, s};
        tile_gemm<double, TN>(c, la, lb, acc, As, Bs);
    }
    const int tx = threadIdx.x % Sh::TX, ty = threadIdx.x / Sh::TX;
#pragma unroll
    for (int i = 0; i < Sh::MI; i++)
#pragma unroll
        for (int j = 0; j < Sh::NJ; j++)
            Rows[(ty + Sh::TY * i) * TN + tx + Sh::TX * j] = -acc[i][j];
    __syncthreads();
    // Lhat_bar = -(G Ybar) - Y S
    const double *Y = A.Z + off + s;
    const double *S = A.YB + off;
    for (int e = threadIdx.x; e < kTM * s; e += kThreads) {
        const int pl = e % kTM, j = e / kTM;
        if (pl >= pm) continue;
        double v = Rows[pl * TN + j];
        for (int k = 0; k < s; k++) v = fma(-Y[(int64_t)k * ld + p0 + pl], S[(int64_t)j * ld + k], v);
        Rows[pl * TN + j] = v;
    }
    __syncthreads();
    // split term of Mbar: P(i, j) = sum_p L_C(p, i) Lhat_bar(p, j)
    const int64_t ss = (int64_t)s * s;
    double *part = A.partial + A.part_off[J] + (int64_t)it.tile * ss;
    const double *Lc = A.L + off + s;
    for (int e = threadIdx.x; e < s * s; e += kThreads) {
        const int i = e % s, j = e / s;
        double v = 0.0;
        for (int pl = 0; pl < pm; pl++) v = fma(Lc[(int64_t)i * ld + p0 + pl], Rows[pl * TN + j], v);
        part[e] = v;
    }
    // Lbar_C rows = Lhat_bar M^T
    const double *Li = A.Linv + A.linv_off[J];
    double *Lb = A.Lb + off + s;
    for (int e = threadIdx.x; e < kTM * s; e += kThreads) {
        const int pl = e % kTM, j = e / kTM;
        if (pl >= pm) continue;
        double v = 0.0;
        for (int k = 0; k < s; k++) v = fma(Rows[pl * TN + k], Li[(int64_t)k * s + j], v);
        Lb[(int64_t)j * ld + p0 + pl] = v;
    }
}

// ---------------------------------------------------------------------------
// Split path of the wide supernodes.  The gather-GEMM G = -A^{-1}(C,C) Ybar
// runs on the tcgen05 kernel (its row exponents: colexpZ, the largest biased
// exponent of each column of A^{-1} on and below the diagonal, where every
// gathered entry is stored); the s-inner products run as separate launches
// of 32 x 32 output blocks so that a level's few tiles still fill the SMs.
// ---------------------------------------------------------------------------
// work (K, 8-column block): a warp per column
__global__ void __launch_bounds__(256) k_adj_colexpz(const AdjDesc *__restrict__ ad, const double *__restrict__ src,
                                                     int *__restrict__ colexpZ, const int2 *__restrict__ work,
                                                     int nwork) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const AdjDesc &A = *ad;
    const int K = work[w].x;
    const int fc = A.super_ptr[K];
    const int s = A.super_ptr[K + 1] - fc;
    const int j = work[w].y * 8 + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (j >= s) return;
    const int64_t ld = A.rowptr[K + 1] - A.rowptr[K];
    const double *Zj = src + A.panel_off[K] + (int64_t)j * ld;
    int e = 0;
    for (int64_t r = j + lane; r < ld; r += 32) e = max(e, bexp(Zj[r]));
#pragma unroll
    for (int o = 16; o; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) colexpZ[fc + j] = e;
}

enum { RP_YBAR = 0, RP_LHB, RP_LBC, RP_MBP, RP_FAC, RP_FABAR, RP_FNBP };

// One 32 x 32 block of
//   RP_YBAR  Ybar = Zbar_{C,K} - Lhat S          (block 0 also stores S)
//   RP_LHB   G   -= Y S                          (G becomes Lhat_bar)
//   RP_LBC   Lbar_{C,K} = Lhat_bar M^T
//   RP_MBP   partial of tile t: P_t(i, j) = sum_{p in t} L_C(p, i) Lhat_bar(p, j),
//            rows i of the item's 32-row block of s
// and of the factorization adjoint (Lb = the working Lbar)
//   RP_FAC   G = A_C = L_C D L_KK^T
//   RP_FABAR Abar_C = Lbar_C D^{-1} M,  M = L_KK^{-1}
//   RP_FNBP  partial of tile t: N_t(i, j) = sum_{p in t} A_C(p, i) Lbar_C(p, j)
// items (K, t, 32-column chunk of s, b): t is the 32-row block of C, or
// for the partials the 64-row tile of C whose slot they fill; b is the
// partials' 32-row block of s.
// Digit planes of the s x s factor B of a row product X B of supernode K, in
// the operand layout of the transposed tcgen05 product (rows = the columns j
// of B, k in 16-steps, the 7 planes of a step one after the other, K-major
// 8 x 8 core matrices), with one exponent per column j.  B by product:
//   RP_YBAR  S, the symmetric cotangent of the diagonal block (also stored
//            in YB's diagonal block, as the product RP_LHB reads it)
//   RP_LHB   S from YB's diagonal block
//   RP_LBC   M^T, M = L_KK^{-1}
//   RP_FAC   D L_KK^T
//   RP_FABAR D^{-1} M
// One CTA per 8 columns, a warp per column; work: (0, K << 8 | column block).
template <int OP>
__global__ void __launch_bounds__(256) k_small_digits(const AdjDesc *__restrict__ ad, const int2 *__restrict__ work,
                                                      int nwork, uint16_t *__restrict__ sd,
                                                      const int64_t *__restrict__ sd_off, int *__restrict__ sdexp) {
    grid_dep_wait();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const AdjDesc &A = *ad;
    const int K = work[w].y >> 8, j = (work[w].y & 0xFF) * 8 + warp;
    const int fc = A.super_ptr[K];
    const int s = A.super_ptr[K + 1] - fc;
    if (j >= s) return;
    const int64_t ld = A.rowptr[K + 1] - A.rowptr[K];
    const int64_t off = A.panel_off[K];
    const int s16 = (s + 15) & ~15;
    const int64_t s64 = (s + 63) / 64 * 64;
    auto val = [&](int k) -> double {
        if (OP == RP_YBAR) {
            if (k == j) return A.Zb[off + (int64_t)j * ld + j];
            return 0.5 * (k > j ? A.Zb[off + (int64_t)j * ld + k] : A.Zb[off + (int64_t)k * ld + j]);
        }
        if (OP == RP_LHB) return A.YB[off + (int64_t)j * ld + k];
        if (OP == RP_LBC) return A.Linv[A.linv_off[K] + (int64_t)k * s + j];
        if (OP == RP_FAC) return k == j ? A.D[fc + k] : (k < j ? A.D[fc + k] * A.L[off + (int64_t)k * ld + j] : 0.0);
        return k >= j ? A.Linv[A.linv_off[K] + (int64_t)j * s + k] / A.D[fc + k] : 0.0;
    };
    int E = 0;
    for (int k = lane; k < s; k += 32) E = max(E, bexp(val(k)));
#pragma unroll
    for (int o = 16; o; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
    if (lane == 0) sdexp[fc + j] = E;
    uint16_t *pu = sd + sd_off[K];
    for (int k = lane; k < s16; k += 32) {
        const double x = k < s ? val(k) : 0.0;
        if (OP == RP_YBAR && k < s) A.YB[off + (int64_t)j * ld + k] = x;
        int d[kDig];
        digits7(x, E, d);
        const int64_t ub = (int64_t)(k / 16) * kDig * s64 * 16 + (j / 8) * 128 + ((k % 16) / 8) * 64 + (j % 8) * 8 + k % 8;
#pragma unroll
        for (int i = 0; i < kDig; i++) pu[i * s64 * 16 + ub] = (uint16_t)f16_of_int(d[i]);
    }
}

// Digit planes of [Ybar, Lhat] (rows p of C, the 2s columns k) for the SYRK
// update of the transposed tcgen05 kernel: per block of 128 rows, per
// 16-step of k the 7 planes of 128 x 16 one after the other (K-major 8 x 8
// core matrices), one exponent per row (at its row position in syexp).  One
// CTA per 32 rows: a warp per 4 rows finds their exponents, then each thread
// cuts 8 consecutive k of one row, a 16-byte store per plane.
// work: (K, 32-row block).
__global__ void __launch_bounds__(256) k_syrk_digits(const AdjDesc *__restrict__ ad, const int2 *__restrict__ work,
                                                     int nwork, uint16_t *__restrict__ sy,
                                                     const int64_t *__restrict__ sy_off, int *__restrict__ syexp) {
    grid_dep_wait();
    __shared__ int rowE[32];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int w = blockIdx.x;
    if (w >= nwork) return;
    const AdjDesc &A = *ad;
    const int K = work[w].x, b = work[w].y;
    const int s = A.super_ptr[K + 1] - A.super_ptr[K];
    const int64_t ld = A.rowptr[K + 1] - A.rowptr[K];
    const int c = (int)(ld - s);
    const int64_t off = A.panel_off[K];
    const int kw = 2 * s, k16 = (kw + 15) / 16 * 16, nst = k16 / 16;
    auto x = [&](int p, int k) -> double {   // [Ybar, Lhat](p, k)
        return k < s ? A.YB[off + (int64_t)k * ld + s + p] : A.LD[off + (int64_t)(k - s) * ld + s + p];
    };
    for (int rr = 0; rr < 4; rr++) {
        const int r = warp * 4 + rr, p = b * 32 + r;
        int E = 0;
        if (p < c)
            for (int k = lane; k < kw; k += 32) E = max(E, bexp(x(p, k)));
#pragma unroll
        for (int o = 16; o; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
        if (lane == 0) {
            rowE[r] = E;
            if (p < c) syexp[A.rowptr[K] + s + p] = E;
        }
    }
    __syncthreads();
    uint16_t *base = sy + sy_off[K];
    for (int e = threadIdx.x; e < 32 * (k16 / 8); e += 256) {
        const int r = e % 32, k0 = (e / 32) * 8, p = b * 32 + r;
        if (p >= c) continue;
        uint32_t h[kDig][4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            int d0[kDig], d1[kDig];
            digits7(k0 + t < kw ? x(p, k0 + t) : 0.0, rowE[r], d0);
            digits7(k0 + t + 1 < kw ? x(p, k0 + t + 1) : 0.0, rowE[r], d1);
#pragma unroll
            for (int i = 0; i < kDig; i++) h[i][t / 2] = f16_of_int(d0[i]) | (f16_of_int(d1[i]) << 16);
        }
        const int t1 = p / 128, r128 = p % 128, st = k0 / 16;
        const int64_t ub = ((int64_t)(t1 * nst + st) * kDig) * 128 * 16 + (r128 / 8) * 128 + ((k0 % 16) / 8) * 64 + (r128 % 8) * 8;
#pragma unroll
        for (int i = 0; i < kDig; i++)
            *reinterpret_cast<uint4 *>(base + ub + (int64_t)i * 128 * 16) = make_uint4(h[i][0], h[i][1], h[i][2], h[i][3]);
    }
}

// The k16 stage of a row-product block: thread (tx, ty) adds rows ty + 16 i
// (i < NI) and columns tx (+ 16 when TWO) of the BM x 32 block.
template <int NI, bool TWO, int BM>
__device__ __forceinline__ void rowprod_stage(const double *As, const double *Bs, int tx, int ty,
                                              double (&acc)[BM / 16][2]) {
#pragma unroll 4
    for (int kk = 0; kk < kTK; kk++) {
        const double b0 = Bs[kk * 32 + tx];
        const double b1 = TWO ? Bs[kk * 32 + tx + 16] : 0.0;
#pragma unroll
        for (int i = 0; i < NI; i++) {
            const double a = As[kk * BM + ty + 16 * i];
            acc[i][0] = fma(a, b0, acc[i][0]);
            if (TWO) acc[i][1] = fma(a, b1, acc[i][1]);
        }
    }
}

template <int OP>
__global__ void __launch_bounds__(kThreads) k_adj_rowprod(const AdjDesc *__restrict__ ad,
                                                          const int4 *__restrict__ items, int nitems) {
    grid_dep_wait();
    constexpr bool kPart = OP == RP_MBP || OP == RP_FNBP;
    constexpr int BM = 32;                  // rows of the output block
    constexpr int MI = BM / 16;
    __shared__ double As[kTK * BM], Bs[kTK * 32];
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const int4 it = items[w];
    const int K = it.x, t = it.y, j0 = it.z * 32, i0 = it.w * 32;
    const int s = A.super_ptr[K + 1] - A.super_ptr[K];
    const int64_t ld = A.rowptr[K + 1] - A.rowptr[K];
    const int c = (int)(ld - s);
    const int64_t off = A.panel_off[K];
    const int rb = kPart ? kTM : BM;          // rows of C per item index t
    const int p0 = t * rb;
    const int pm = c - p0 < rb ? (c - p0 > 0 ? c - p0 : 0) : rb;
    const int nj = s - j0 < 32 ? s - j0 : 32;
    const int mrows = kPart ? (s - i0 < 32 ? s - i0 : 32) : pm;
    const int kdim = kPart ? pm : s;
    const int fc = A.super_ptr[K];
    const double *Zb = A.Zb + off;
    const double *S = A.YB + off;      // S(k, j) = S[j * ld + k]
    auto sym = [&](int k, int j) -> double {   // S from the cotangent's lower diagonal block
        if (k == j) return Zb[(int64_t)j * ld + j];
        return 0.5 * (k > j ? Zb[(int64_t)j * ld + k] : Zb[(int64_t)k * ld + j]);
    };
    auto a_at = [&](int r, int k) -> double {
        if (OP == RP_YBAR) return A.LD[off + (int64_t)k * ld + s + p0 + r];
        if (OP == RP_LHB) return A.Z[off + (int64_t)k * ld + s + p0 + r];
        if (OP == RP_LBC) return A.G[off + (int64_t)k * ld + s + p0 + r];
        if (OP == RP_MBP) return A.L[off + (int64_t)(i0 + r) * ld + s + p0 + k];
        if (OP == RP_FAC) return A.L[off + (int64_t)k * ld + s + p0 + r] * A.D[fc + k];
        if (OP == RP_FABAR) return A.Lb[off + (int64_t)k * ld + s + p0 + r];
        return A.G[off + (int64_t)(i0 + r) * ld + s + p0 + k];
    };
    auto b_at = [&](int k, int jl) -> double {
        const int j = j0 + jl;
        if (OP == RP_YBAR) return sym(k, j);
        if (OP == RP_LHB) return S[(int64_t)j * ld + k];
        if (OP == RP_LBC) return A.Linv[A.linv_off[K] + (int64_t)k * s + j];
        if (OP == RP_MBP) return A.G[off + (int64_t)j * ld + s + p0 + k];
        if (OP == RP_FAC) return k == j ? 1.0 : (k < j ? A.L[off + (int64_t)k * ld + j] : 0.0);   // L_KK(j, k)
        if (OP == RP_FABAR) return k >= j ? A.Linv[A.linv_off[K] + (int64_t)j * s + k] / A.D[fc + k] : 0.0;
        return A.Lb[off + (int64_t)j * ld + s + p0 + k];
    };
    // thread (tx, ty) owns rows ty + 16 i and columns tx + 16 j of the block.
    // A warp holds rows 2 warp, 2 warp + 1 (+ 16 i): the row blocks with no
    // row of the item, and the second column half when nj <= 16, are skipped
    // (warp-uniform), which for the narrow supernodes is most of the block.
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int wrow = 2 * (threadIdx.x / 32);
    const int ni = mrows > wrow ? min((mrows - wrow + 15) / 16, MI) : 0;
    const int sel = ni * 2 + (nj > 16 ? 1 : 0);
    double acc[MI][2];
#pragma unroll
    for (int i = 0; i < MI; i++) acc[i][0] = acc[i][1] = 0.0;
    for (int k0 = 0; k0 < kdim; k0 += kTK) {
        __syncthreads();
        for (int e = threadIdx.x; e < kTK * BM; e += kThreads) {
            const int r = e % BM, k = k0 + e / BM;
            As[e] = (r < mrows && k < kdim) ? a_at(r, k) : 0.0;
        }
        for (int e = threadIdx.x; e < kTK * 32; e += kThreads) {
            const int kk = e % kTK, jl = e / kTK, k = k0 + kk;
            Bs[kk * 32 + jl] = (k < kdim && jl < nj) ? b_at(k, jl) : 0.0;
        }
        __syncthreads();
        switch (sel) {
        case 2: rowprod_stage<1, false, BM>(As, Bs, tx, ty, acc); break;
        case 3: rowprod_stage<1, true, BM>(As, Bs, tx, ty, acc); break;
        case 4: rowprod_stage<2, false, BM>(As, Bs, tx, ty, acc); break;
        case 5: rowprod_stage<2, true, BM>(As, Bs, tx, ty, acc); break;
        case 6: if constexpr (MI >= 3) rowprod_stage<3, false, BM>(As, Bs, tx, ty, acc); break;
        case 7: if constexpr (MI >= 3) rowprod_stage<3, true, BM>(As, Bs, tx, ty, acc); break;
        case 8: if constexpr (MI >= 4) rowprod_stage<4, false, BM>(As, Bs, tx, ty, acc); break;
        case 9: if constexpr (MI >= 4) rowprod_stage<4, true, BM>(As, Bs, tx, ty, acc); break;
        default: break;
        }
    }
#pragma unroll
    for (int i = 0; i < MI; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int r = ty + 16 * i, q = tx + 16 * j;
            if (r >= mrows || q >= nj) continue;
            if (kPart) {
                const int64_t ss = (int64_t)s * s;
                A.partial[A.part_off[K] + (int64_t)t * ss + (int64_t)(j0 + q) * s + i0 + r] = acc[i][j];
                continue;
            }
            const int64_t e = off + (int64_t)(j0 + q) * ld + s + p0 + r;
            if (OP == RP_YBAR) A.YB[e] = A.Zb[e] - acc[i][j];
            else if (OP == RP_LHB) A.G[e] -= acc[i][j];
            else if (OP == RP_LBC) A.Lb[e] = acc[i][j];
            else if (OP == RP_FAC) A.G[e] = acc[i][j];
            else A.Ab[e] = acc[i][j];
        }
    if (OP == RP_YBAR && t == 0)
        for (int e = threadIdx.x; e < s * nj; e += kThreads) {
            const int k = e % s, j = j0 + e / s;
            A.YB[off + (int64_t)j * ld + k] = sym(k, j);
        }
}

// ---------------------------------------------------------------------------
// factorization adjoint
// ---------------------------------------------------------------------------
template <int TN>
__global__ void __launch_bounds__(kThreads) k_fadj_pull(const AdjDesc *__restrict__ ad,
                                                        const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    using Sh = Shape<TN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *As = reinterpret_cast<double *>(smem_raw);
    double *Bs = As + kTK * (kTM > TN ? kTM : TN);
    double *Rows = Bs + kTK * TN;
    __shared__ int64_t tile_cb[kTM], tile_rb[kTM];
    __shared__ int s_last;
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const Item it = items[w];
    const int J = it.K;
    const int fc = A.super_ptr[J];
    const int s = A.super_ptr[J + 1] - fc;
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const int c = (int)(ld - s);
    const int p0 = it.tile * kTM;
    const int pm = c - p0 < kTM ? c - p0 : kTM;
    const int64_t pos0 = A.rowptr[J] + s;
    const int64_t off = A.panel_off[J];
    for (int e = threadIdx.x; e < kTM; e += kThreads) {
        const int p = p0 + e;
        tile_cb[e] = p < c ? A.colbase[pos0 + p] : 0;
        tile_rb[e] = p < c ? A.relbase[pos0 + p] : 0;
    }
    double acc[Sh::MI][Sh::NJ];
#pragma unroll
    for (int i = 0; i < Sh::MI; i++)
#pragma unroll
        for (int j = 0; j < Sh::NJ; j++) acc[i][j] = 0.0;
    if (pm > 0) {
        LoadGather<double, TN, true> la{A.Ab, A.colbase + pos0, A.relbase + pos0, A.relidx, tile_cb, tile_rb, p0, c};
        LoadColMajor<double, TN> lb{A.L + off + s, ld, c, s};
        tile_gemm<double, TN>(c, la, lb, acc, As, Bs);
    }
    const int tx = threadIdx.x % Sh::TX, ty = threadIdx.x / Sh::TX;
#pragma unroll
    for (int i = 0; i < Sh::MI; i++)
#pragma unroll
        for (int j = 0; j < Sh::NJ; j++) Rows[(ty + Sh::TY * i) * TN + tx + Sh::TX * j] = acc[i][j];
    __syncthreads();
    const double *D = A.D + fc;
    const double *Lc = A.L + off + s;
    double *Lb = A.Lb + off + s;
    for (int e = threadIdx.x; e < kTM * s; e += kThreads) {
        const int pl = e % kTM, k = e / kTM;
        if (pl >= pm) continue;
        Lb[(int64_t)k * ld + p0 + pl] -= Rows[pl * TN + k] * D[k];
    }
    double *part = A.partial + A.part_off[J] + (int64_t)it.tile * s * s;
    for (int k = threadIdx.x; k < s; k += kThreads) {
        double v = 0.0;
        for (int pl = 0; pl < pm; pl++) v = fma(Lc[(int64_t)k * ld + p0 + pl], Rows[pl * TN + k], v);
        part[k] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&A.counter[J], 1) == it.ntiles - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double *part0 = A.partial + A.part_off[J];
    for (int k = threadIdx.x; k < s; k += kThreads) {
        double v = 0.0;
        for (int t = 0; t < it.ntiles; t++) v += ldcg(part0 + (int64_t)t * s * s + k);
        A.Db[fc + k] -= 0.5 * v;
    }
    if (threadIdx.x == 0) A.counter[J] = 0;
}

// k_fadj_pull for a wide supernode whose gather-GEMM ran on the tensor
// cores: G = -Abar(C,C) L_C with every gathered entry counted once, so the
// doubled diagonal adds Abar(C[p], C[p]) L_C(p, :) here.  A warp per column.
__global__ void __launch_bounds__(256) k_fadj_pull_tc(const AdjDesc *__restrict__ ad,
                                                      const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    __shared__ double dg[kTM];
    __shared__ int s_last;
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const Item it = items[w];
    const int J = it.K;
    const int fc = A.super_ptr[J];
    const int s = A.super_ptr[J + 1] - fc;
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const int c = (int)(ld - s);
    const int p0 = it.tile * kTM;
    const int pm = c - p0 < kTM ? (c - p0 > 0 ? c - p0 : 0) : kTM;
    const int64_t pos0 = A.rowptr[J] + s;
    const int64_t off = A.panel_off[J];
    for (int e = threadIdx.x; e < kTM; e += blockDim.x) {
        const int p = p0 + e;
        dg[e] = e < pm ? A.Ab[A.colbase[pos0 + p] + A.relidx[A.relbase[pos0 + p] + p]] : 0.0;
    }
    __syncthreads();
    const double *D = A.D + fc;
    const double *Lc = A.L + off + s;
    const double *G = A.G + off + s;
    double *Lb = A.Lb + off + s;
    double *part = A.partial + A.part_off[J] + (int64_t)it.tile * s * s;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int k = warp; k < s; k += 8) {
        double v = 0.0;
        for (int pl = lane; pl < pm; pl += 32) {
            const int64_t e = (int64_t)k * ld + p0 + pl;
            const double r = fma(dg[pl], Lc[e], -G[e]);   // (Abar(C,C) L_C)(p, k), diagonal doubled
            Lb[e] -= r * D[k];
            v = fma(Lc[e], r, v);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[k] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&A.counter[J], 1) == it.ntiles - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double *part0 = A.partial + A.part_off[J];
    for (int k = threadIdx.x; k < s; k += blockDim.x) {
        double v = 0.0;
        for (int t = 0; t < it.ntiles; t++) v += ldcg(part0 + (int64_t)t * s * s + k);
        A.Db[fc + k] -= 0.5 * v;
    }
    if (threadIdx.x == 0) A.counter[J] = 0;
}

// Abar_C rows = Lbar_C D^{-1} L_JJ^{-1}; split Nbar = A_C^T Lbar_C
template <int TN>
__global__ void __launch_bounds__(kThreads) k_fadj_trsm(const AdjDesc *__restrict__ ad,
                                                        const Item *__restrict__ items, int nitems) {
    grid_dep_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *Ar = reinterpret_cast<double *>(smem_raw);    // [TM][TN] A_C rows
    double *Br = Ar + kTM * TN;                            // [TM][TN] Lbar_C rows
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const Item it = items[w];
    const int J = it.K;
    const int fc = A.super_ptr[J];
    const int s = A.super_ptr[J + 1] - fc;
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const int c = (int)(ld - s);
    const int p0 = it.tile * kTM;
    const int pm = c - p0 < kTM ? c - p0 : kTM;
    const int64_t off = A.panel_off[J];
    const double *L = A.L + off;
    const double *D = A.D + fc;
    const double *Li = A.Linv + A.linv_off[J];
    const double *Lb = A.Lb + off + s;
    double *Ab = A.Ab + off + s;
    for (int e = threadIdx.x; e < kTM * s; e += kThreads) {
        const int pl = e % kTM, j = e / kTM;
        double a = 0.0;
        if (pl < pm) {
            // A_C(p, j) = sum_{k <= j} L_C(p, k) D_k L_JJ(j, k)
            for (int k = 0; k <= j; k++) {
                const double ljk = (k == j) ? 1.0 : L[(int64_t)k * ld + j];
                a = fma(L[(int64_t)k * ld + s + p0 + pl] * D[k], ljk, a);
            }
            Br[pl * TN + j] = Lb[(int64_t)j * ld + p0 + pl];
        } else {
            Br[pl * TN + j] = 0.0;
        }
        Ar[pl * TN + j] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kTM * s; e += kThreads) {  // Abar_C = (Lbar_C D^{-1}) M
        const int pl = e % kTM, j = e / kTM;
        if (pl >= pm) continue;
        double v = 0.0;
        for (int k = j; k < s; k++) v = fma(Br[pl * TN + k] / D[k], Li[(int64_t)j * s + k], v);
        Ab[(int64_t)j * ld + p0 + pl] = v;
    }
    const int64_t ss = (int64_t)s * s;
    double *part = A.partial + A.part_off[J] + (int64_t)it.tile * ss;
    for (int e = threadIdx.x; e < s * s; e += kThreads) {    // Nbar partial = A_C^T Lbar_C
        const int i = e % s, j = e / s;
        double v = 0.0;
        for (int pl = 0; pl < pm; pl++) v = fma(Ar[pl * TN + i], Br[pl * TN + j], v);
        part[e] = v;
    }
}

__global__ void k_gather_vals(const int64_t *__restrict__ pos, const double *__restrict__ src,
                              int64_t n, double *__restrict__ dst) {
    grid_dep_wait();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[pos[e]];
}


// ---------------------------------------------------------------------------
// Per-supernode s x s steps of both adjoints, batched over a tree level and
// spread over many CTAs.  Scratch per supernode J: 4 s x s slots at
// 4 * linv_off[J] (selinv: Mbar, W, T1; factorization: Nbar, T2, N, U).
// ---------------------------------------------------------------------------
enum { OP_SEL_T1 = 0, OP_SEL_W, OP_SEL_LB, OP_FAC_T2, OP_FAC_U, OP_FAC_T3, OP_FAC_G1, OP_FAC_G2 };
constexpr int kFinChunk = 1024;   // entries of an s x s block per item of the partial sums

// C (16 x 16 tile) of an s x s product; items (J, tile), tiles row-major over
// ceil(s/16)^2 (16 CTAs per 64 columns: the top levels hold one or two
// supernodes).  Q = 1: a CTA of 256 threads per tile, one output each; Q = 4
// (levels with fewer tiles than SMs): four CTAs of 64 threads per tile, an
// 8 x 8 quarter each, so that the FP64 work spreads over four times the SMs.
// k staged kGK at a time (one stage up to s = 128: one round of load latency).
constexpr int kGT = 16;
constexpr int kGK = 128;
template <int Q, int op>
__global__ void __launch_bounds__(256) k_adj_gemm(const AdjDesc *__restrict__ ad, const int2 *__restrict__ items,
                                                  int nitems) {
    grid_dep_wait();
    constexpr int GT = Q == 1 ? kGT : kGT / 2;   // output tile side of the CTA
    constexpr int NT = GT * GT;                  // threads
    __shared__ double As[GT][kGK + 1], Bs[kGK][GT + 1];
    const int w = blockIdx.x / Q, qd = blockIdx.x % Q;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const int J = items[w].x;
    const int s = A.super_ptr[J + 1] - A.super_ptr[J];
    const int nt = (s + kGT - 1) / kGT;
    const int i0 = (items[w].y / nt) * kGT + (Q == 1 ? 0 : (qd / 2) * GT);
    const int j0 = (items[w].y % nt) * kGT + (Q == 1 ? 0 : (qd % 2) * GT);
    if (i0 >= s || j0 >= s) return;
    const int64_t ss = (int64_t)s * s;
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const double *M = A.Linv + A.linv_off[J];             // M(i, k) = M[k*s + i]
    double *F = A.fin + 4 * A.linv_off[J];
    const double *S = A.YB + A.panel_off[J];              // S(k, j) = S[j*ld + k]
    const double *LJ = A.L + A.panel_off[J];              // L_JJ(i, k) = LJ[k*ld + i], unit lower
    const double *LbJ = A.Lb + A.panel_off[J];
    auto a_at = [&](int i, int k) -> double {
        switch (op) {
        case OP_SEL_T1: return M[(int64_t)k * s + i];                 // M
        case OP_SEL_W: return F[(int64_t)k * s + i];                  // Mbar
        case OP_SEL_LB: return M[(int64_t)i * s + k];                 // M^T
        case OP_FAC_T2: return F[(int64_t)k * s + i];                 // Nbar
        case OP_FAC_U: return F[2 * ss + (int64_t)i * s + k];         // N^T
        case OP_FAC_T3: return k == i ? 1.0 : (k > i ? LJ[(int64_t)i * ld + k] : 0.0);  // L_JJ^T
        case OP_FAC_G1: return F[(int64_t)k * s + i];                 // P
        default: return M[(int64_t)i * s + k];                        // M^T
        }
    };
    auto b_at = [&](int k, int j) -> double {
        switch (op) {
        case OP_SEL_T1: return S[(int64_t)j * ld + k];                // S
        case OP_SEL_W: return M[(int64_t)k * s + j];                  // M^T
        case OP_SEL_LB: return F[ss + (int64_t)j * s + k];            // W
        case OP_FAC_T2: return F[2 * ss + (int64_t)k * s + j];        // N^T
        case OP_FAC_U: return F[ss + (int64_t)j * s + k];             // T2
        case OP_FAC_T3: return k > j ? LbJ[(int64_t)j * ld + k] : 0.0;  // Lbar_JJ, strictly lower
        case OP_FAC_G1: return M[(int64_t)j * s + k];                 // M
        default: return F[ss + (int64_t)j * s + k];                   // P M
        }
    };
    const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;
    // a warp holds 32 / GT rows of the tile: warps past s skip the products,
    // and the last k stage stops at s
    const bool wact = i0 + (32 / GT) * (int)(threadIdx.x / 32) < s;
    // every product has a triangular factor (M = L_JJ^{-1} and L_JJ are lower
    // triangular): the k-range of the tile stops at its last row or column, or
    // starts at its first -- half the FP64 work on average
    int klo = 0, khi = s;
    switch (op) {
    case OP_SEL_T1: khi = min(s, i0 + GT); break;   // M(i, k): k <= i
    case OP_SEL_W: khi = min(s, j0 + GT); break;    // M(j, k): k <= j
    case OP_SEL_LB: klo = i0; break;                // M(k, i): k >= i
    case OP_FAC_T2: klo = j0; break;                // N(j, k) = M(k, j) / D_k: k >= j
    case OP_FAC_U: khi = min(s, i0 + GT); break;    // N(k, i) = M(i, k) / D_i: k <= i
    case OP_FAC_T3: klo = i0; break;                // L_JJ(k, i): k >= i
    case OP_FAC_G1: klo = j0; break;                // M(k, j): k >= j
    default: klo = i0; break;                       // M(k, i): k >= i
    }
    double acc = 0.0;
    for (int k0 = klo; k0 < khi; k0 += kGK) {
        const int kn = khi - k0 < kGK ? khi - k0 : kGK;
        __syncthreads();
#pragma unroll 4
        for (int e = threadIdx.x; e < GT * kn; e += NT) {
            const int r = e % GT, q = e / GT;
            As[r][q] = i0 + r < s ? a_at(i0 + r, k0 + q) : 0.0;
            Bs[q][r] = j0 + r < s ? b_at(k0 + q, j0 + r) : 0.0;
        }
        __syncthreads();
        if (wact) {
            double a2 = 0.0;   // two chains: half the FMA latency per k
            int q = 0;
#pragma unroll 4
            for (; q + 1 < kn; q += 2) {
                acc = fma(As[ty][q], Bs[q][tx], acc);
                a2 = fma(As[ty][q + 1], Bs[q + 1][tx], a2);
            }
            if (q < kn) acc = fma(As[ty][q], Bs[q][tx], acc);
            acc += a2;
        }
    }
    double *Lb = A.Lb + A.panel_off[J];
    const int i = i0 + ty, j = j0 + tx;
    if (i >= s || j >= s) return;
    const double x = acc;
    switch (op) {
    case OP_SEL_T1: F[2 * ss + (int64_t)j * s + i] = x; break;               // T1
    case OP_SEL_W: F[ss + (int64_t)j * s + i] = x; break;                    // W
    case OP_SEL_LB: Lb[(int64_t)j * ld + i] = i > j ? -x : 0.0; break;      // Lbar_JJ
    case OP_FAC_T2: F[ss + (int64_t)j * s + i] = x; break;                   // T2
    case OP_FAC_U: F[3 * ss + (int64_t)j * s + i] = -x; break;               // Ubar
    case OP_FAC_T3:                                                          // P
        F[(int64_t)j * s + i] = i > j ? x / A.D[A.super_ptr[J] + j] : (i == j ? A.Db[A.super_ptr[J] + i] : 0.0);
        break;
    case OP_FAC_G1: F[ss + (int64_t)j * s + i] = x; break;                   // P M
    default: F[2 * ss + (int64_t)j * s + i] = x; break;                      // G = M^T P M
    }
}

// A row product X B (c x s by s x s) of a wide supernode as 16 x 16 output
// tiles (Q = 1, 256 threads) or their 8 x 8 quarters (Q = 4, 64 threads),
// for the levels whose tcgen05 product launch would run only a few CTAs (the
// top of the tree): the FP64 work spreads over every SM.  OP as in
// k_adj_rowprod (YBAR, LHB, LBC, FAC, FABAR); items (K, tile), tiles
// row-major over ceil(max(c, 1) / 16) x ceil(s / 16); the tiles of row 0 of
// RP_YBAR also store S.
template <int Q, int OP>
__global__ void __launch_bounds__(256) k_adj_rowgemm(const AdjDesc *__restrict__ ad, const int2 *__restrict__ items,
                                                     int nitems) {
    grid_dep_wait();
    constexpr int GT = Q == 1 ? kGT : kGT / 2;
    constexpr int NT = GT * GT;
    __shared__ double As[GT][kGK + 1], Bs[kGK][GT + 1];
    const int w = blockIdx.x / Q, qd = blockIdx.x % Q;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const int K = items[w].x;
    const int fc = A.super_ptr[K];
    const int s = A.super_ptr[K + 1] - fc;
    const int64_t ld = A.rowptr[K + 1] - A.rowptr[K];
    const int c = (int)(ld - s);
    const int64_t off = A.panel_off[K];
    const int ntj = (s + kGT - 1) / kGT;
    const int ti = items[w].y / ntj;
    const int i0 = ti * kGT + (Q == 1 ? 0 : (qd / 2) * GT);
    const int j0 = (items[w].y % ntj) * kGT + (Q == 1 ? 0 : (qd % 2) * GT);
    if (j0 >= s) return;
    const double *Zb = A.Zb + off;
    auto sym = [&](int k, int j) -> double {   // S from the cotangent's lower diagonal block
        if (k == j) return Zb[(int64_t)j * ld + j];
        return 0.5 * (k > j ? Zb[(int64_t)j * ld + k] : Zb[(int64_t)k * ld + j]);
    };
    if (OP == RP_YBAR && ti == 0 && qd < 2)   // S into YB's diagonal block, this tile's columns
        for (int e = threadIdx.x; e < s * GT; e += NT) {
            const int k = e % s, j = j0 + e / s;
            if (j < s) A.YB[off + (int64_t)j * ld + k] = sym(k, j);
        }
    if (i0 >= c) return;
    auto a_at = [&](int i, int k) -> double {   // X(i, k), i a row of C
        const int64_t e = off + (int64_t)k * ld + s + i;
        if (OP == RP_YBAR) return A.LD[e];
        if (OP == RP_LHB) return A.Z[e];
        if (OP == RP_LBC) return A.G[e];
        if (OP == RP_FAC) return A.L[e] * A.D[fc + k];
        return A.Lb[e];
    };
    auto b_at = [&](int k, int j) -> double {   // B(k, j)
        if (OP == RP_YBAR) return sym(k, j);
        if (OP == RP_LHB) return A.YB[off + (int64_t)j * ld + k];
        if (OP == RP_LBC) return A.Linv[A.linv_off[K] + (int64_t)k * s + j];
        if (OP == RP_FAC) return k == j ? 1.0 : (k < j ? A.L[off + (int64_t)k * ld + j] : 0.0);   // L_KK(j, k)
        return k >= j ? A.Linv[A.linv_off[K] + (int64_t)j * s + k] / A.D[fc + k] : 0.0;
    };
    // triangular factors: M^T (LBC) and L_KK^T (FAC) vanish for k > j,
    // D^{-1} M (FABAR) for k < j
    int klo = 0, khi = s;
    if (OP == RP_LBC || OP == RP_FAC) khi = min(s, j0 + GT);
    if (OP == RP_FABAR) klo = j0;
    const int tx = threadIdx.x % GT, ty = threadIdx.x / GT;
    const bool wact = i0 + (32 / GT) * (int)(threadIdx.x / 32) < c;
    double acc = 0.0;
    for (int k0 = klo; k0 < khi; k0 += kGK) {
        const int kn = khi - k0 < kGK ? khi - k0 : kGK;
        __syncthreads();
#pragma unroll 4
        for (int e = threadIdx.x; e < GT * kn; e += NT) {
            const int r = e % GT, q = e / GT;
            As[r][q] = i0 + r < c ? a_at(i0 + r, k0 + q) : 0.0;
            Bs[q][r] = j0 + r < s ? b_at(k0 + q, j0 + r) : 0.0;
        }
        __syncthreads();
        if (wact) {
            double a2 = 0.0;
            int q = 0;
#pragma unroll 4
            for (; q + 1 < kn; q += 2) {
                acc = fma(As[ty][q], Bs[q][tx], acc);
                a2 = fma(As[ty][q + 1], Bs[q + 1][tx], a2);
            }
            if (q < kn) acc = fma(As[ty][q], Bs[q][tx], acc);
            acc += a2;
        }
    }
    const int i = i0 + ty, j = j0 + tx;
    if (i >= c || j >= s) return;
    const int64_t e = off + (int64_t)j * ld + s + i;
    if (OP == RP_YBAR) A.YB[e] = A.Zb[e] - acc;
    else if (OP == RP_LHB) A.G[e] -= acc;
    else if (OP == RP_LBC) A.Lb[e] = acc;
    else if (OP == RP_FAC) A.G[e] = acc;
    else A.Ab[e] = acc;
}

// selinv adjoint: Mbar = sum of the tile partials + 2 D^{-1} T1 (T1 = M S);
// items (J, chunk of kFinChunk entries | ntiles << 16)
__global__ void __launch_bounds__(256) k_adj_sel_mbar(const AdjDesc *__restrict__ ad,
                                                      const int2 *__restrict__ items, int nitems) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const int J = items[w].x, chunk = items[w].y & 0xFFFF, ntiles = items[w].y >> 16;
    const int fc = A.super_ptr[J];
    const int s = A.super_ptr[J + 1] - fc;
    const int64_t ss = (int64_t)s * s;
    double *__restrict__ F = A.fin + 4 * A.linv_off[J];
    const double *__restrict__ part = A.partial + A.part_off[J];
    const int64_t e1 = (int64_t)(chunk + 1) * kFinChunk < ss ? (int64_t)(chunk + 1) * kFinChunk : ss;
    for (int64_t e = (int64_t)chunk * kFinChunk + threadIdx.x; e < e1; e += blockDim.x) {
        const int i = (int)(e % s);
        double v = 0.0;
        for (int t = 0; t < ntiles; t++) v += part[t * ss + e];
        F[e] = v + 2.0 * F[2 * ss + e] / A.D[fc + i];
    }
}

// selinv adjoint: Dbar_k = -(M S M^T)_kk / D_k^2 = -sum_a T1(k, a) M(k, a) / D_k^2;
// grid (supernodes, kFinY): 32 values of k per pass, the eight warps take
// every eighth a, their sums added in a fixed order
__global__ void __launch_bounds__(256) k_adj_sel_dbar(const AdjDesc *__restrict__ ad,
                                                      const int *__restrict__ js, int nj) {
    grid_dep_wait();
    __shared__ double red[8][33];
    const int w = blockIdx.x;
    if (w >= nj) return;
    const AdjDesc &A = *ad;
    const int J = js[w];
    const int fc = A.super_ptr[J];
    const int s = A.super_ptr[J + 1] - fc;
    const int64_t ss = (int64_t)s * s;
    const double *__restrict__ M = A.Linv + A.linv_off[J];
    const double *__restrict__ T1 = A.fin + 4 * A.linv_off[J] + 2 * ss;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int kb = blockIdx.y; kb * 32 < s; kb += gridDim.y) {
        const int k = kb * 32 + lane;
        double v = 0.0;
        if (k < s)
            for (int a = warp; a < s; a += 8) v = fma(T1[(int64_t)a * s + k], M[(int64_t)a * s + k], v);
        red[warp][lane] = v;
        __syncthreads();
        if (warp == 0 && k < s) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < 8; q++) t += red[q][lane];
            A.Db[fc + k] = -t / (A.D[fc + k] * A.D[fc + k]);
        }
        __syncthreads();
    }
}

// factorization adjoint: Nbar = sum of the tile partials; N = M^T D^{-1};
// items as in k_adj_sel_mbar
__global__ void __launch_bounds__(256) k_fadj_nbar(const AdjDesc *__restrict__ ad,
                                                   const int2 *__restrict__ items, int nitems) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const AdjDesc &A = *ad;
    const int J = items[w].x, chunk = items[w].y & 0xFFFF, ntiles = items[w].y >> 16;
    const int fc = A.super_ptr[J];
    const int s = A.super_ptr[J + 1] - fc;
    const int64_t ss = (int64_t)s * s;
    double *__restrict__ F = A.fin + 4 * A.linv_off[J];
    const double *__restrict__ M = A.Linv + A.linv_off[J];
    const double *__restrict__ part = A.partial + A.part_off[J];
    const int64_t e1 = (int64_t)(chunk + 1) * kFinChunk < ss ? (int64_t)(chunk + 1) * kFinChunk : ss;
    for (int64_t e = (int64_t)chunk * kFinChunk + threadIdx.x; e < e1; e += blockDim.x) {
        const int i = (int)(e % s), j = (int)(e / s);
        double v = 0.0;
        for (int t = 0; t < ntiles; t++) v += part[t * ss + e];
        F[e] = v;
        F[2 * ss + e] = M[(int64_t)i * s + j] / A.D[fc + j];   // N(i, j) = M(j, i) / D_j
    }
}

// factorization adjoint: U = D L^T gives Dbar_i += sum_{j>=i} Ubar(i,j) L(j,i),
// Lbar(j,i) += Ubar(i,j) D_i (j > i); grid (supernodes, kFinY), the sums as
// in k_adj_sel_dbar
__global__ void __launch_bounds__(256) k_fadj_ubar(const AdjDesc *__restrict__ ad,
                                                   const int *__restrict__ js, int nj) {
    grid_dep_wait();
    __shared__ double red[8][33];
    const int w = blockIdx.x;
    if (w >= nj) return;
    const AdjDesc &A = *ad;
    const int J = js[w];
    const int fc = A.super_ptr[J];
    const int s = A.super_ptr[J + 1] - fc;
    const int64_t ss = (int64_t)s * s;
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const double *__restrict__ U = A.fin + 4 * A.linv_off[J] + 3 * ss;
    const double *__restrict__ L = A.L + A.panel_off[J];
    double *__restrict__ Lb = A.Lb + A.panel_off[J];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int ib = blockIdx.y; ib * 32 < s; ib += gridDim.y) {
        const int i = ib * 32 + lane;
        double v = 0.0;
        if (i < s)
            for (int j = i + 1 + warp; j < s; j += 8) v = fma(U[(int64_t)j * s + i], L[(int64_t)i * ld + j], v);
        red[warp][lane] = v;
        __syncthreads();
        if (warp == 0 && i < s) {
            double t = U[(int64_t)i * s + i];
#pragma unroll
            for (int q = 0; q < 8; q++) t += red[q][lane];
            A.Db[fc + i] += t;
        }
        __syncthreads();
    }
    for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < ss; e += (int64_t)gridDim.y * blockDim.x) {
        const int j = (int)(e % s), i = (int)(e / s);
        if (j > i) Lb[(int64_t)i * ld + j] += U[(int64_t)j * s + i] * A.D[fc + i];
    }
}

// factorization adjoint: reverse of the dense LDL^T of J's diagonal block in
// closed form.  With X = L^{-1} dA L^{-T} one has dD = diag(X) and
// dL = L stril(X) D^{-1}, so dloss = <P, X> with
//   P = stril(L^T Lbar D^{-1}) + diag(Dbar),
// and the full-matrix gradient is G = L^{-T} P L^{-1} = M^T P M (M = L_JJ^{-1};
// three s x s products in k_adj_gemm).  The stored lower entries of the
// symmetric block get G(i,j) + G(j,i) below the diagonal, G(i,i) on it.
// Grid (supernodes, kFinY).
__global__ void __launch_bounds__(256) k_fadj_fold(const AdjDesc *__restrict__ ad,
                                                   const int *__restrict__ js, int nj) {
    grid_dep_wait();
    const int w = blockIdx.x;
    if (w >= nj) return;
    const AdjDesc &A = *ad;
    const int J = js[w];
    const int s = A.super_ptr[J + 1] - A.super_ptr[J];
    const int64_t ld = A.rowptr[J + 1] - A.rowptr[J];
    const int64_t ss = (int64_t)s * s;
    const double *__restrict__ G = A.fin + 4 * A.linv_off[J] + 2 * ss;
    double *__restrict__ Ab = A.Ab + A.panel_off[J];
    for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < ss; e += (int64_t)gridDim.y * blockDim.x) {
        const int i = (int)(e % s), k = (int)(e / s);
        Ab[(int64_t)k * ld + i] = i > k ? G[(int64_t)k * s + i] + G[(int64_t)i * s + k]
                                        : (i == k ? G[(int64_t)k * s + i] : 0.0);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int TN> static size_t lhbar_smem() {
    return sizeof(double) * ((size_t)kTK * (kTM > TN ? kTM : TN) + kTK * TN + (size_t)kTM * TN);
}
template <int TN> static size_t trsm_smem() { return sizeof(double) * 2 * (size_t)kTM * TN; }

static cudaError_t configure_adjoint() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define CFG(K, TN, SZ) if (e == cudaSuccess) e = cudaFuncSetAttribute(K<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SZ<TN>())
    CFG(k_adj_lhbar, 8, lhbar_smem); CFG(k_adj_lhbar, 16, lhbar_smem); CFG(k_adj_lhbar, 32, lhbar_smem);
    CFG(k_adj_lhbar, 64, lhbar_smem); CFG(k_adj_lhbar, 128, lhbar_smem);
    CFG(k_fadj_pull, 8, lhbar_smem); CFG(k_fadj_pull, 16, lhbar_smem); CFG(k_fadj_pull, 32, lhbar_smem);
    CFG(k_fadj_pull, 64, lhbar_smem); CFG(k_fadj_pull, 128, lhbar_smem);
    CFG(k_fadj_trsm, 8, trsm_smem); CFG(k_fadj_trsm, 16, trsm_smem); CFG(k_fadj_trsm, 32, trsm_smem);
    CFG(k_fadj_trsm, 64, trsm_smem); CFG(k_fadj_trsm, 128, trsm_smem);
#undef CFG
    done = e == cudaSuccess;
    return e;
}

template <template <int> class KF> struct Dummy {};

template <int OP>
static void launch_gemm_op(AdjData *a, int64_t g0, int n, cudaStream_t st) {
    if (n < kNumSMs) k_adj_gemm<4, OP><<<4 * n, kGT * kGT / 4, 0, st>>>(a->d_desc, a->d_gitems + g0, n);
    else k_adj_gemm<1, OP><<<n, kGT * kGT, 0, st>>>(a->d_desc, a->d_gitems + g0, n);
}

static void launch_level_gemm(AdjData *a, int op, int li, cudaStream_t st) {
    const int64_t g0 = a->g_lptr[li], g1 = a->g_lptr[li + 1];
    const int n = (int)(g1 - g0);
    if (n <= 0) return;
    switch (op) {
    case OP_SEL_T1: launch_gemm_op<OP_SEL_T1>(a, g0, n, st); break;
    case OP_SEL_W: launch_gemm_op<OP_SEL_W>(a, g0, n, st); break;
    case OP_SEL_LB: launch_gemm_op<OP_SEL_LB>(a, g0, n, st); break;
    case OP_FAC_T2: launch_gemm_op<OP_FAC_T2>(a, g0, n, st); break;
    case OP_FAC_U: launch_gemm_op<OP_FAC_U>(a, g0, n, st); break;
    case OP_FAC_T3: launch_gemm_op<OP_FAC_T3>(a, g0, n, st); break;
    case OP_FAC_G1: launch_gemm_op<OP_FAC_G1>(a, g0, n, st); break;
    default: launch_gemm_op<OP_FAC_G2>(a, g0, n, st); break;
    }
    note_launch();
}

static void launch_bucket(int kind, int b, const AdjDesc *d, const Item *items, int n, cudaStream_t st) {
    if (n <= 0) return;
#define L3(KERN, TN, SZ) KERN<TN><<<n, kThreads, SZ<TN>(), st>>>(d, items, n)
    switch (kind * 8 + b) {
    case 0: L3(k_adj_lhbar, 8, lhbar_smem); break;
    case 1: L3(k_adj_lhbar, 16, lhbar_smem); break;
    case 2: L3(k_adj_lhbar, 32, lhbar_smem); break;
    case 3: L3(k_adj_lhbar, 64, lhbar_smem); break;
    case 4: L3(k_adj_lhbar, 128, lhbar_smem); break;
    case 8: L3(k_fadj_pull, 8, lhbar_smem); break;
    case 9: L3(k_fadj_pull, 16, lhbar_smem); break;
    case 10: L3(k_fadj_pull, 32, lhbar_smem); break;
    case 11: L3(k_fadj_pull, 64, lhbar_smem); break;
    case 12: L3(k_fadj_pull, 128, lhbar_smem); break;
    case 16: L3(k_fadj_trsm, 8, trsm_smem); break;
    case 17: L3(k_fadj_trsm, 16, trsm_smem); break;
    case 18: L3(k_fadj_trsm, 32, trsm_smem); break;
    case 19: L3(k_fadj_trsm, 64, trsm_smem); break;
    default: L3(k_fadj_trsm, 128, trsm_smem); break;
    }
#undef L3
    note_launch();
}

void adjoint_release(void *p) {
    AdjData *a = static_cast<AdjData *>(p);
    if (!a) return;
    auto fr = [](void *q) { if (q) cudaFree(q); };
    fr(a->d_items); fr(a->d_lhat); fr(a->d_linv);
    fr(a->d_gitems); fr(a->d_citems); fr(a->d_js); fr(a->d_cz); fr(a->d_vitems);
    fr(a->YB); fr(a->Zb); fr(a->Lbw); fr(a->Ab); fr(a->fin); fr(a->d_desc); fr(a->d_pdesc);
    fr(a->V);
    fr(a->d_sm); fr(a->d_wd); fr(a->d_row); fr(a->d_rg); fr(a->d_mbp); fr(a->d_dig); fr(a->d_tcdesc); fr(a->cy);
    fr(a->d_pr); fr(a->d_sdw); fr(a->sd); fr(a->d_sd_off); fr(a->sdexp); fr(a->d_pdp);
    fr(a->d_syw); fr(a->d_sy); fr(a->d_vn); fr(a->sy); fr(a->d_sy_off); fr(a->syexp); fr(a->d_sydesc);
    if (a->g_sel) cudaGraphExecDestroy(a->g_sel);
    if (a->g_fac) cudaGraphExecDestroy(a->g_fac);
    a->tcs.release();
    a->tcn.release();
    delete a;
}

template <typename X>
static int upl(X **d, const std::vector<X> &h) {
    *d = nullptr;
    if (cudaMalloc((void **)d, sizeof(X) * std::max<size_t>(1, h.size())) != cudaSuccess) return SELINV_ERR_OOM;
    if (!h.empty() && cudaMemcpy(*d, h.data(), sizeof(X) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SELINV_ERR_CUDA;
    return SELINV_OK;
}

static int adj_build(selinv_plan_s *plan) {
    if (!plan->factor) plan->factor = new FactorData();
    int rc = factor_tables(plan);
    if (rc) return rc;
    FactorData *f = plan->factor;
    if (f->adj) return SELINV_OK;
    const PlanData &p = plan->data;
    AdjData *a = new AdjData();
    // per level (deepest first) items sorted by bucket; 64-row panel tiles
    a->lvl_bucket_ptr.push_back(0);
    for (int l = p.nlevels - 1; l >= 0; l--) {
        for (int b = 0; b < kNumBuckets; b++) {
            for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                const int32_t J = p.level_list[e];
                if (bucket_of(p.super_ptr[J + 1] - p.super_ptr[J]) != b) continue;
                for (int t = 0; t < p.ntiles[J]; t++) a->items.push_back({0, J, t, p.ntiles[J]});
            }
            a->lvl_bucket_ptr.push_back((int)a->items.size());
        }
    }
    a->g_lptr.assign(1, 0); a->c_lptr.assign(1, 0); a->j_lptr.assign(1, 0); a->cz_lptr.assign(1, 0);
    a->v_lptr.assign(1, 0);
    for (int l = p.nlevels - 1; l >= 0; l--) {      // deepest first, like every list here
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t J = p.level_list[e];
            const int s = p.super_ptr[J + 1] - p.super_ptr[J];
            const int nt = (s + kGT - 1) / kGT;
            for (int t = 0; t < nt * nt; t++) a->gitems.push_back(make_int2(J, t));
            const int nch = (int)(((int64_t)s * s + kFinChunk - 1) / kFinChunk);
            for (int ch = 0; ch < nch; ch++) a->citems.push_back(make_int2(J, ch | (p.ntiles[J] << 16)));
            a->js.push_back(J);
            for (int jb = 0; jb < (s + 7) / 8; jb++) a->cz_work.push_back(make_int2(J, jb));
            const int64_t cJ = p.rowptr[J + 1] - p.rowptr[J] - s;
            const int nvt = (int)((cJ + kVB - 1) / kVB);
            for (int ti = 0; ti < nvt; ti++)
                for (int tj = 0; tj <= ti; tj++) a->vitems.push_back(make_int4(J, ti, tj, 0));
        }
        a->cz_lptr.push_back((int64_t)a->cz_work.size());
        a->v_lptr.push_back((int64_t)a->vitems.size());
        a->g_lptr.push_back((int64_t)a->gitems.size());
        a->c_lptr.push_back((int64_t)a->citems.size());
        a->j_lptr.push_back((int64_t)a->js.size());
    }
    for (int32_t K = 0; K < p.ns; K++) a->linv_work.push_back(make_int2(0, K));
    a->lhat_bptr.push_back(0);
    for (int b = 0; b < kNumBuckets; b++) {
        for (int32_t K = 0; K < p.ns; K++) {
            const int s = p.super_ptr[K + 1] - p.super_ptr[K];
            const int64_t c = p.rowptr[K + 1] - p.rowptr[K] - s;
            if (c == 0 || bucket_of(s) != b) continue;
            for (int t = 0; t < p.ntiles[K]; t++) a->lhat_items.push_back({0, K, t, p.ntiles[K]});
        }
        a->lhat_bptr.push_back((int)a->lhat_items.size());
    }
    if (cudaMalloc((void **)&a->V, 8 * (size_t)std::max<int64_t>(f->u_off[p.ns], 1)) != cudaSuccess) {
        adjoint_release(a);
        return SELINV_ERR_OOM;
    }
    if ((rc = upl(&a->d_items, a->items)) || (rc = upl(&a->d_lhat, a->lhat_items)) ||
        (rc = upl(&a->d_linv, a->linv_work)) ||
        (rc = upl(&a->d_gitems, a->gitems)) || (rc = upl(&a->d_citems, a->citems)) || (rc = upl(&a->d_js, a->js)) ||
        (rc = upl(&a->d_cz, a->cz_work)) || (rc = upl(&a->d_vitems, a->vitems))) {
        adjoint_release(a);
        return rc;
    }
    const size_t nz = (size_t)std::max<int64_t>(p.nnz, 1);
    if (cudaMalloc((void **)&a->YB, 8 * nz) || cudaMalloc((void **)&a->Zb, 8 * nz) ||
        cudaMalloc((void **)&a->Lbw, 8 * nz) || cudaMalloc((void **)&a->Ab, 8 * nz) ||
        cudaMalloc((void **)&a->fin, 8 * (size_t)std::max<int64_t>(4 * p.linv_total, 1)) ||
        cudaMalloc((void **)&a->d_desc, sizeof(AdjDesc)) || cudaMalloc((void **)&a->d_pdesc, sizeof(ProbDesc))) {
        adjoint_release(a);
        return SELINV_ERR_OOM;
    }
    f->adj = a;
    return SELINV_OK;
}

static AdjDesc make_adesc(selinv_plan_s *plan, const double *L, const double *D, const double *Z,
                          double *Lb, double *Db) {
    const PlanData &p = plan->data;
    FactorData *f = plan->factor;
    AdjData *a = static_cast<AdjData *>(f->adj);
    Workspace &w = plan->ws[0];
    AdjDesc h;
    h.super_ptr = p.d_super_ptr; h.rowptr = p.d_rowptr; h.rows = p.d_rows; h.panel_off = p.d_panel_off;
    h.colbase = p.d_colbase; h.relbase = p.d_relbase; h.relidx = p.d_relidx;
    h.linv_off = p.d_linv_off; h.part_off = p.d_part_off;
    h.L = L; h.D = D; h.Z = Z;
    h.LD = static_cast<const double *>(w.LD);
    h.Linv = static_cast<const double *>(w.Linv);
    h.Zb = a->Zb; h.YB = a->YB; h.Lb = Lb; h.Db = Db; h.Ab = a->Ab;
    h.partial = static_cast<double *>(w.partial);
    h.counter = w.counter;
    h.fin = a->fin;
    h.sparent = p.d_sparent;
    h.v_off = f->d_uoff;
    h.chpos = f->d_chpos;
    h.V = a->V;
    h.G = static_cast<double *>(w.work);
    return h;
}

// L_KK^{-1}, Dinv and Lhat of every supernode (the forward normalization)
static int adj_normalize(selinv_plan_s *plan, const void *L, const void *D, cudaStream_t st) {
    AdjData *a = static_cast<AdjData *>(plan->factor->adj);
    ProbDesc pd = make_desc(plan->data, plan->ws[0], SELINV_F64, L, D, nullptr, false);
    cudaMemcpyAsync(a->d_pdesc, &pd, sizeof(pd), cudaMemcpyHostToDevice, st);
    if (!a->tcn.launches.empty()) {
        // the forward's own normalization launches (Lhat of the wide supernodes on the tensor cores)
        for (const Launch &Ln : a->tcn.launches)
            if (Ln.kind == KL_LINV || Ln.kind == KL_DINV || Ln.kind == KL_LINV_DIGITS || Ln.kind == KL_LHAT_OZ ||
                Ln.kind == KL_LHAT) {
                launch_with(a->tcn, Ln, a->d_pdesc, st);
                note_launch();
            }
        return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
    }
    launch_linv(SELINV_F64, a->d_pdesc, a->d_linv, (int)a->linv_work.size(), 1, st);
    note_launch();
    for (int b = 0; b < kNumBuckets; b++) {
        const int n = a->lhat_bptr[b + 1] - a->lhat_bptr[b];
        if (n > 0) {
            launch_lhat(SELINV_F64, b, a->d_pdesc, a->d_lhat + a->lhat_bptr[b], n, st);
            note_launch();
        }
    }
    return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}

// The per-level lists of the selected-inversion adjoint for the current
// options: wide supernodes are those the forward contracts on tcgen05.
static int adj_split(selinv_plan_s *plan) {
    AdjData *a = static_cast<AdjData *>(plan->factor->adj);
    const PlanData &p = plan->data;
    const selinv_opts &o = p.opts;
    // (at least 8 columns: narrower supernodes keep the fused kernels, whose
    // one CTA per tile wastes less than 32-column blocks would, unless C has
    // kAdjWideC rows or more: there one fused CTA per tile would run the whole
    // gather over C alone).  Any tensor engine of the forward means tcgen05
    // here: the reverse passes have no mma.sync variant.
    const int key = o.fast_contraction != 0 ? std::max(8, o.oz_min_s) : 0;
    if (key == a->split_key) return SELINV_OK;
    auto fr = [](void *q) { if (q) cudaFree(q); };
    fr(a->d_sm); fr(a->d_wd); fr(a->d_row); fr(a->d_rg); fr(a->d_mbp); fr(a->d_dig);
    fr(a->d_pr); fr(a->d_sdw); fr(a->sd); fr(a->d_sd_off);
    fr(a->d_syw); fr(a->d_sy); fr(a->d_vn); fr(a->sy); fr(a->d_sy_off);
    a->d_sm = a->d_wd = nullptr; a->d_row = a->d_mbp = nullptr; a->d_dig = nullptr; a->d_rg = nullptr;
    a->d_pr = nullptr; a->d_sdw = nullptr; a->sd = nullptr; a->d_sd_off = nullptr;
    a->d_syw = nullptr; a->d_sy = nullptr; a->d_vn = nullptr; a->sy = nullptr; a->d_sy_off = nullptr;
    a->sy_work.clear(); a->sy_items.clear(); a->vn_items.clear();
    a->sy_wlptr.assign(1, 0); a->sy_lptr.assign(1, 0); a->vn_lptr.assign(1, 0);
    std::vector<int64_t> sy_off(p.ns + 1, 0);
    int64_t sy_max = 0;
    a->tcs.release();
    a->tcs.launches.clear();
    a->tcn.release();
    a->tcn.launches.clear();
    a->sm_items.clear(); a->wd_items.clear(); a->row_items.clear(); a->mbp_items.clear(); a->dig_work.clear();
    a->rg_items.clear(); a->rg_lptr.assign(1, 0);
    a->pr_items.clear(); a->sd_work.clear();
    a->sm_bptr.assign(1, 0); a->wd_lptr.assign(1, 0); a->row_lptr.assign(1, 0); a->mbp_lptr.assign(1, 0); a->dig_lptr.assign(1, 0);
    a->pr_lptr.assign(1, 0); a->sd_lptr.assign(1, 0);
    std::vector<int64_t> sd_off(p.ns + 1, 0);
    a->tc_launch.assign(p.nlevels, {});
    auto wide = [&](int s, int64_t c) { return key > 0 && (s >= key || c >= kAdjWideC); };
    auto wideK = [&](int32_t J) {
        const int s = p.super_ptr[J + 1] - p.super_ptr[J];
        return wide(s, p.rowptr[J + 1] - p.rowptr[J] - s);
    };
    for (int l = p.nlevels - 1; l >= 0; l--) {
        for (int b = 0; b < kNumBuckets; b++) {
            for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
                const int32_t J = p.level_list[e];
                const int s = p.super_ptr[J + 1] - p.super_ptr[J];
                if (wideK(J) || bucket_of(s) != b) continue;
                for (int t = 0; t < p.ntiles[J]; t++) a->sm_items.push_back({0, J, t, p.ntiles[J]});
            }
            a->sm_bptr.push_back((int)a->sm_items.size());
        }
        // the level's row products on the FP64 kernel when none of its wide
        // supernodes is wider than kRowSimtS columns, else all on tcgen05 (one
        // launch per product: a second, narrower launch would add its latency)
        int wmax = 0;
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t J = p.level_list[e];
            if (wideK(J)) wmax = std::max(wmax, p.super_ptr[J + 1] - p.super_ptr[J]);
        }
        const bool simt = wmax <= kRowSimtS;
        double fma = 0.0;   // multiply-adds of one of the level's row products
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t J = p.level_list[e];
            if (!wideK(J)) continue;
            const double sj = p.super_ptr[J + 1] - p.super_ptr[J];
            fma += (double)(p.rowptr[J + 1] - p.rowptr[J] - (int64_t)sj) * sj * sj;
        }
        const bool small = !simt && fma < kSmallProdFma;
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t J = p.level_list[e];
            const int s = p.super_ptr[J + 1] - p.super_ptr[J];
            if (!wideK(J)) continue;
            const int64_t c = p.rowptr[J + 1] - p.rowptr[J] - s;
            const int nch = (s + 31) / 32;
            for (int t = 0; t < p.ntiles[J]; t++) a->wd_items.push_back({0, J, t, p.ntiles[J]});
            if (simt)   // (one block even without C: block 0 of RP_YBAR also stores S)
                for (int b = 0; b < std::max<int64_t>(1, (c + 31) / 32); b++)
                    for (int ch = 0; ch < nch; ch++) a->row_items.push_back(make_int4(J, b, ch, 0));
            for (int t = 0; t < p.ntiles[J]; t++)
                for (int ch = 0; ch < nch; ch++)
                    for (int h = 0; h < (s + 31) / 32; h++) a->mbp_items.push_back(make_int4(J, t, ch, h));
            if (c > 0)
                for (int jb = 0; jb < (s + 7) / 8; jb++) a->dig_work.push_back(make_int2(0, (J << 8) | jb));
            if (small) {
                const int ntj = (s + kGT - 1) / kGT, nti = (int)std::max<int64_t>(1, (c + kGT - 1) / kGT);
                for (int t = 0; t < nti * ntj; t++) a->rg_items.push_back(make_int2(J, t));
            } else if (!simt) {
                for (int64_t t = 0; t < (c + kTcWideRows - 1) / kTcWideRows; t++) a->pr_items.push_back({0, J, (int)t, 1});
                for (int jb = 0; jb < (s + 7) / 8; jb++) a->sd_work.push_back(make_int2(0, (J << 8) | jb));
            }
        }
        a->wd_lptr.push_back((int64_t)a->wd_items.size());
        a->row_lptr.push_back((int64_t)a->row_items.size());
        a->rg_lptr.push_back((int64_t)a->rg_items.size());
        a->mbp_lptr.push_back((int64_t)a->mbp_items.size());
        a->dig_lptr.push_back((int64_t)a->dig_work.size());
        a->pr_lptr.push_back((int64_t)a->pr_items.size());
        a->sd_lptr.push_back((int64_t)a->sd_work.size());
        // the update matrices: SYRK items for the wide supernodes, k_adj_vupd
        // tiles for the rest; digit offsets restart at every level
        int64_t lev_off = 0;
        for (int64_t e = p.level_ptr[l]; e < p.level_ptr[l + 1]; e++) {
            const int32_t J = p.level_list[e];
            const int s = p.super_ptr[J + 1] - p.super_ptr[J];
            const int64_t c = p.rowptr[J + 1] - p.rowptr[J] - s;
            if (c == 0) continue;
            if (!wide(s, c)) {
                const int nvt = (int)((c + kVB - 1) / kVB);
                for (int ti = 0; ti < nvt; ti++)
                    for (int tj = 0; tj <= ti; tj++) a->vn_items.push_back(make_int4(J, ti, tj, 0));
                continue;
            }
            const int64_t n1 = (c + 127) / 128, n2 = (c + kTcWideRows - 1) / kTcWideRows;
            const int64_t k16 = (2 * (int64_t)s + 15) / 16 * 16;
            sy_off[J] = lev_off;
            lev_off += n1 * 128 * k16 * 7;
            for (int64_t t1 = 0; t1 < n1; t1++)
                for (int64_t t2 = 0; t2 < n2 && t2 * kTcWideRows <= t1 * 128 + 127; t2++)
                    a->sy_items.push_back({0, J, (int)(t1 * n2 + t2), 1});
            for (int64_t b = 0; b < (c + 31) / 32; b++) a->sy_work.push_back(make_int2(J, (int)b));
        }
        sy_max = std::max(sy_max, lev_off);
        a->sy_wlptr.push_back((int64_t)a->sy_work.size());
        a->sy_lptr.push_back((int64_t)a->sy_items.size());
        a->vn_lptr.push_back((int64_t)a->vn_items.size());
    }
    for (int32_t J = 0; J < p.ns; J++) {
        const int64_t s = p.super_ptr[J + 1] - p.super_ptr[J];
        sd_off[J + 1] = sd_off[J] + (wideK(J) ? 7 * ((s + 63) / 64 * 64) * ((s + 15) / 16 * 16) : 0);
    }
    int rc;
    if ((rc = upl(&a->d_sm, a->sm_items)) || (rc = upl(&a->d_wd, a->wd_items)) || (rc = upl(&a->d_row, a->row_items)) ||
        (rc = upl(&a->d_rg, a->rg_items)) ||
        (rc = upl(&a->d_mbp, a->mbp_items)) || (rc = upl(&a->d_dig, a->dig_work)) ||
        (rc = upl(&a->d_pr, a->pr_items)) || (rc = upl(&a->d_sdw, a->sd_work)) || (rc = upl(&a->d_sd_off, sd_off)) ||
        (rc = upl(&a->d_syw, a->sy_work)) || (rc = upl(&a->d_sy, a->sy_items)) || (rc = upl(&a->d_vn, a->vn_items)) ||
        (rc = upl(&a->d_sy_off, sy_off)))
        return rc;
    if (sy_max > 0 && cudaMalloc((void **)&a->sy, sizeof(uint16_t) * (size_t)sy_max) != cudaSuccess)
        return SELINV_ERR_OOM;
    if (!a->syexp && cudaMalloc((void **)&a->syexp, sizeof(int) * (size_t)std::max<int64_t>(p.rowptr[p.ns], 1)) != cudaSuccess)
        return SELINV_ERR_OOM;
    if (!a->d_sydesc && cudaMalloc((void **)&a->d_sydesc, sizeof(ProbDesc)) != cudaSuccess) return SELINV_ERR_OOM;
    if (sd_off[p.ns] > 0 && cudaMalloc((void **)&a->sd, sizeof(uint16_t) * (size_t)sd_off[p.ns]) != cudaSuccess)
        return SELINV_ERR_OOM;
    if (!a->sdexp && cudaMalloc((void **)&a->sdexp, sizeof(int) * (size_t)std::max(p.n, 1)) != cudaSuccess)
        return SELINV_ERR_OOM;
    if (!a->d_pdp && cudaMalloc((void **)&a->d_pdp, 5 * sizeof(ProbDesc)) != cudaSuccess) return SELINV_ERR_OOM;
    if (!a->dig_work.empty()) {
        // the forward's level schedule supplies the tcgen05 items of every
        // level (row tiles, column tiles, k-splits) and their reductions, built
        // for exactly the wide supernodes (as the selection, whatever width;
        // a subset selection of the forward does not apply here)
        const ProbDesc pd = make_desc(p, plan->ws[0], SELINV_F64, nullptr, nullptr, nullptr, false);
        std::vector<uint8_t> sel(p.ns, 0);
        for (int32_t J = 0; J < p.ns; J++) sel[J] = wideK(J) ? 1 : 0;
        sel.swap(plan->data.active);
        const int fcon = plan->data.opts.fast_contraction, ozm = plan->data.opts.oz_min_s;
        plan->data.opts.fast_contraction = 1;
        plan->data.opts.oz_min_s = kOzMinS;
        rc = build_schedule(a->tcs, {&p}, {pd}, SELINV_SCHED_LEVEL, false);
        plan->data.opts.oz_min_s = ozm;
        sel.swap(plan->data.active);
        // and the normalization of every supernode, as the forward runs it
        sel.clear();
        sel.swap(plan->data.active);
        if (!rc) rc = build_schedule(a->tcn, {&p}, {pd}, SELINV_SCHED_LEVEL, false);
        sel.swap(plan->data.active);
        plan->data.opts.fast_contraction = fcon;
        if (rc) return rc;
        for (int e = 0; e < (int)a->tcs.launches.size(); e++) {
            const Launch &L = a->tcs.launches[e];
            if ((L.kind == KL_SELINV_TC || L.kind == KL_TC_REDUCE) && L.level >= 0 && L.level < p.nlevels)
                a->tc_launch[p.nlevels - 1 - L.level].push_back(e);
        }
    }
    if (!a->d_tcdesc && cudaMalloc((void **)&a->d_tcdesc, sizeof(ProbDesc)) != cudaSuccess) return SELINV_ERR_OOM;
    if (!a->cy && cudaMalloc((void **)&a->cy, sizeof(int) * (size_t)std::max(p.n, 1)) != cudaSuccess)
        return SELINV_ERR_OOM;
    a->split_key = key;
    a->gen++;
    return SELINV_OK;
}

// options that may change between calls without changing the lists
static void adj_refresh(selinv_plan_s *plan) {
    AdjData *a = static_cast<AdjData *>(plan->factor->adj);
    a->tcs.spin_limit = plan->data.opts.spin_limit;
    a->tcn.spin_limit = plan->data.opts.spin_limit;
}

static int adj_prepare(selinv_plan_s *plan) {
    int rc = ensure_device(plan->data);
    if (rc) return rc;
    if ((rc = adj_build(plan))) return rc;
    if (plan->ws.empty()) plan->ws.resize(1);
    if ((rc = plan->ws[0].ensure(plan->data, SELINV_F64))) return rc;
    return configure_adjoint() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}

}  // namespace selinv

using namespace selinv;

// One row product X B of the level's wide supernodes on the transposed
// tcgen05 kernel: the digit planes of B, then the product (descriptor pd of
// d_pdp: the panel X, the output and its mode).
template <int OP>
static void row_product(AdjData *a, int pd, int li, cudaStream_t st) {
    const int r0 = (int)a->row_lptr[li], r1 = (int)a->row_lptr[li + 1];
    if (r1 > r0) {   // the narrower wide supernodes: 32 x 32 blocks on the FP64 kernel
        k_adj_rowprod<OP><<<r1 - r0, kThreads, 0, st>>>(a->d_desc, a->d_row + r0, r1 - r0);
        note_launch();
    }
    const int g0 = (int)a->rg_lptr[li], g1 = (int)a->rg_lptr[li + 1];
    if (g1 > g0) {   // the top levels: 16 x 16 tiles (8 x 8 quarters) on the FP64 kernel
        if (g1 - g0 < kNumSMs)
            k_adj_rowgemm<4, OP><<<4 * (g1 - g0), kGT * kGT / 4, 0, st>>>(a->d_desc, a->d_rg + g0, g1 - g0);
        else
            k_adj_rowgemm<1, OP><<<g1 - g0, kGT * kGT, 0, st>>>(a->d_desc, a->d_rg + g0, g1 - g0);
        note_launch();
    }
    const int q0 = (int)a->sd_lptr[li], q1 = (int)a->sd_lptr[li + 1];
    if (q1 > q0) {
        k_small_digits<OP><<<q1 - q0, 256, 0, st>>>(a->d_desc, a->d_sdw + q0, q1 - q0, a->sd, a->d_sd_off, a->sdexp);
        note_launch();
    }
    const int t0 = (int)a->pr_lptr[li], t1 = (int)a->pr_lptr[li + 1];
    if (t1 > t0) {
        launch_lhat_tcw(a->d_pdp + pd, a->d_pr + t0, t1 - t0, a->tcs.spin_limit, st);
        note_launch();
    }
}

// Issues body(st) through a CUDA graph captured on the first call and replayed
// afterwards.  The per-level launches of the reverse passes take only the
// plan's own device buffers as arguments (the caller's pointers reach them
// through descriptors uploaded before the graph runs), so one capture serves
// every call until the lists (key) or the workspace (ws) change.  A stream
// that cannot be captured -- the legacy default stream, or one the caller is
// capturing already -- runs body(st) directly.
template <class F>
static int run_captured(cudaGraphExec_t &exec, int &nlaunch, long long &key, const void *&ws, long long want_key,
                        const void *want_ws, cudaStream_t st, F body) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st == nullptr || st == cudaStreamLegacy || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone) {
        body(st);
        return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
    }
    if (!exec || key != want_key || ws != want_ws) {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        const int64_t n0 = selinv_launch_count();
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SELINV_ERR_CUDA;
        body(st);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        nlaunch = (int)(selinv_launch_count() - n0);
        note_launch(-nlaunch);   // captured, not yet issued
        if (e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return SELINV_ERR_CUDA;
        }
        if (programmatic_edges(g) != cudaSuccess) {
            cudaGraphDestroy(g);
            return SELINV_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            exec = nullptr;
            return SELINV_ERR_CUDA;
        }
        key = want_key;
        ws = want_ws;
    }
    note_launch(nlaunch);
    return cudaGraphLaunch(exec, st) == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}

extern "C" int selinv_adjoint(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D,
                              const void *Z, const void *Zbar, void *Lbar, void *Dbar, void *stream) {
    NvtxRange nvtx_range("selinv_adjoint");
    if (!plan) return SELINV_ERR_INVALID_ARG;
    if (dtype != SELINV_F64) return SELINV_ERR_UNSUPPORTED;
    if (plan->data.ns == 0) return SELINV_OK;
    if (!L || !D || !Z || !Zbar || !Lbar || !Dbar) return SELINV_ERR_INVALID_ARG;
    if (!plan->data.active.empty()) return SELINV_ERR_UNSUPPORTED;   // needs every block of A^{-1}
    int rc = adj_prepare(plan);
    if (rc) return rc;
    if ((rc = adj_split(plan))) return rc;
    adj_refresh(plan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    plan->last_stream = st;
    const PlanData &p = plan->data;
    AdjData *a = static_cast<AdjData *>(plan->factor->adj);
    if ((rc = adj_normalize(plan, L, D, st))) return rc;
    const size_t bytes = 8 * (size_t)p.nnz;
    cudaMemcpyAsync(a->Zb, Zbar, bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(Lbar, 0, bytes, st);
    cudaMemsetAsync(Dbar, 0, 8 * (size_t)p.n, st);
    AdjDesc h = make_adesc(plan, static_cast<const double *>(L), static_cast<const double *>(D),
                           static_cast<const double *>(Z), static_cast<double *>(Lbar),
                           static_cast<double *>(Dbar));
    cudaMemcpyAsync(a->d_desc, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    k_adj_fold<<<dim3(p.ns, kFinY), 256, 0, st>>>(a->d_desc, p.ns);
    note_launch();
    FactorData *f = plan->factor;
    cudaMemsetAsync(a->V, 0, 8 * (size_t)std::max<int64_t>(f->u_off[p.ns], 1), st);
    Workspace &w = plan->ws[0];
    if (!a->dig_work.empty()) {
        // tcgen05 gather-GEMM: A^{-1}(C,C) from Z, B = Ybar (digit planes of
        // YB), output G; row exponents from Z's columns
        ProbDesc pd = make_desc(p, w, SELINV_F64, L, D, const_cast<void *>(Z), false);
        pd.LD = a->YB;
        pd.Yout = w.work;
        pd.colexpY = a->cy;
        cudaMemcpyAsync(a->d_tcdesc, &pd, sizeof(pd), cudaMemcpyHostToDevice, st);
        // the row products: Ybar = Zbar_{C,K} - Lhat S, G -= Y S (G becomes
        // Lhat_bar), Lbar_{C,K} = Lhat_bar M^T
        ProbDesc base = make_desc(p, w, SELINV_F64, L, D, const_cast<void *>(Z), false);
        base.linvd = a->sd;
        base.linvd_off = a->d_sd_off;
        base.linvexp = a->sdexp;
        ProbDesc pdp[3] = {base, base, base};
        pdp[0].L = w.LD; pdp[0].LD = a->YB; pdp[0].Yout = a->Zb; pdp[0].prod_op = 2;
        pdp[1].L = Z; pdp[1].LD = w.work; pdp[1].prod_op = 1;
        pdp[2].L = w.work; pdp[2].LD = Lbar; pdp[2].prod_op = 0;
        cudaMemcpyAsync(a->d_pdp, pdp, sizeof(pdp), cudaMemcpyHostToDevice, st);
        // the update V_K -= sym(Ybar Lhat^T): B = [Lhat, Ybar] from the panels
        // LD and YB, A = the digit planes of [Ybar, Lhat], out V (offsets u_off)
        ProbDesc sy = base;
        sy.L = w.LD;
        sy.Z = a->YB;
        sy.Yout = a->V;
        sy.part_off = f->d_uoff;
        sy.linvd = a->sy;
        sy.linvd_off = a->d_sy_off;
        sy.linvexp = a->syexp;
        cudaMemcpyAsync(a->d_sydesc, &sy, sizeof(sy), cudaMemcpyHostToDevice, st);
        const int ncz = (int)a->cz_work.size();
        k_adj_colexpz<<<ncz, 256, 0, st>>>(a->d_desc, static_cast<const double *>(Z), w.colexpZ, a->d_cz, ncz);
        note_launch();
    }
    const int nl = p.nlevels;
    auto levels = [&](cudaStream_t st) {
        for (int li = 0; li < nl; li++) {  // deepest level first
            // the children's update matrices complete Zbar on K's panel and start V_K
            for (int r = 0; r < f->npass; r++) {
                const int64_t x0 = f->asm_lptr[li * f->npass + r], x1 = f->asm_lptr[li * f->npass + r + 1];
                if (x1 > x0) { k_adj_asm<<<(int)(x1 - x0), 256, 0, st>>>(a->d_desc, f->d_asm + x0, (int)(x1 - x0)); note_launch(); }
            }
            const int i0 = a->sm_bptr[li * kNumBuckets], i1 = a->sm_bptr[(li + 1) * kNumBuckets];
            if (i1 > i0) { k_adj_ybar<<<i1 - i0, 256, 0, st>>>(a->d_desc, a->d_sm + i0, i1 - i0); note_launch(); }
            const int m0 = (int)a->mbp_lptr[li], m1 = (int)a->mbp_lptr[li + 1];
            row_product<RP_YBAR>(a, 0, li, st);
            const int64_t v0 = a->vn_lptr[li], v1 = a->vn_lptr[li + 1];
            if (v1 > v0) { k_adj_vupd<<<(int)(v1 - v0), 256, 0, st>>>(a->d_desc, a->d_vn + v0, (int)(v1 - v0)); note_launch(); }
            const int64_t y0 = a->sy_wlptr[li], y1 = a->sy_wlptr[li + 1];
            if (y1 > y0) {
                k_syrk_digits<<<(int)(y1 - y0), 256, 0, st>>>(a->d_desc, a->d_syw + y0, (int)(y1 - y0), a->sy, a->d_sy_off, a->syexp);
                note_launch();
            }
            const int64_t z0 = a->sy_lptr[li], z1 = a->sy_lptr[li + 1];
            if (z1 > z0) {
                launch_syrk_tcw(a->d_sydesc, a->d_sy + z0, (int)(z1 - z0), a->tcs.spin_limit, st);
                note_launch();
            }
            const int d0 = (int)a->dig_lptr[li], d1 = (int)a->dig_lptr[li + 1];
            if (d1 > d0) {
                launch_lhat_digits(a->d_tcdesc, a->d_dig + d0, d1 - d0, st);
                note_launch();
                for (int e : a->tc_launch[li]) {
                    launch_with(a->tcs, a->tcs.launches[e], a->d_tcdesc, st);
                    note_launch();
                }
            }
            for (int b = 0; b < kNumBuckets; b++) {
                const int b0 = a->sm_bptr[li * kNumBuckets + b], b1 = a->sm_bptr[li * kNumBuckets + b + 1];
                launch_bucket(0, b, a->d_desc, a->d_sm + b0, b1 - b0, st);
            }
            row_product<RP_LHB>(a, 1, li, st);
            if (m1 > m0) {
                k_adj_rowprod<RP_MBP><<<m1 - m0, kThreads, 0, st>>>(a->d_desc, a->d_mbp + m0, m1 - m0);
                note_launch();
            }
            row_product<RP_LBC>(a, 2, li, st);
            // per-supernode s x s steps, batched over the level
            const int64_t c0 = a->c_lptr[li], c1 = a->c_lptr[li + 1];
            const int64_t j0 = a->j_lptr[li], j1 = a->j_lptr[li + 1];
            launch_level_gemm(a, OP_SEL_T1, li, st);
            if (c1 > c0) { k_adj_sel_mbar<<<(int)(c1 - c0), 256, 0, st>>>(a->d_desc, a->d_citems + c0, (int)(c1 - c0)); note_launch(); }
            launch_level_gemm(a, OP_SEL_W, li, st);
            launch_level_gemm(a, OP_SEL_LB, li, st);
            if (j1 > j0) { k_adj_sel_dbar<<<dim3((int)(j1 - j0), kFinY), 256, 0, st>>>(a->d_desc, a->d_js + j0, (int)(j1 - j0)); note_launch(); }
        }
    };
    return run_captured(a->g_sel, a->g_sel_n, a->g_sel_key, a->g_sel_ws, a->gen, w.colexpZ, st, levels);
}

extern "C" int selinv_factor_adjoint(selinv_plan plan, selinv_dtype dtype, const void *L, const void *D,
                                     const void *Lbar, const void *Dbar, void *Abar_vals, void *stream) {
    NvtxRange nvtx_range("selinv_factor_adjoint");
    if (!plan || !plan->factor) return SELINV_ERR_INVALID_ARG;
    if (dtype != SELINV_F64) return SELINV_ERR_UNSUPPORTED;
    if (plan->data.ns == 0) return SELINV_OK;
    if (!L || !D || !Lbar || !Dbar || (plan->factor->nnzA > 0 && !Abar_vals)) return SELINV_ERR_INVALID_ARG;
    int rc = adj_prepare(plan);
    if (rc) return rc;
    if ((rc = adj_split(plan))) return rc;
    adj_refresh(plan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    plan->last_stream = st;
    const PlanData &p = plan->data;
    FactorData *f = plan->factor;
    AdjData *a = static_cast<AdjData *>(f->adj);
    if ((rc = adj_normalize(plan, L, D, st))) return rc;
    const size_t bytes = 8 * (size_t)p.nnz;
    // working copies: Lbar -> Lbw, Dbar -> YB's first n slots (YB is free here)
    cudaMemcpyAsync(a->Lbw, Lbar, bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a->YB, Dbar, 8 * (size_t)p.n, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(a->Ab, 0, bytes, st);
    AdjDesc h = make_adesc(plan, static_cast<const double *>(L), static_cast<const double *>(D), nullptr,
                           a->Lbw, a->YB);
    cudaMemcpyAsync(a->d_desc, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    Workspace &w = plan->ws[0];
    const bool tc = !a->dig_work.empty();
    if (tc) {
        // tcgen05 gather-GEMM of the wide supernodes: A^{-1}(C,C) -> the
        // finished Abar of the ancestors, B = L_C (digit planes of L, once),
        // output G; Abar's column exponents follow level by level
        ProbDesc pd = make_desc(p, w, SELINV_F64, L, D, a->Ab, false);
        pd.LD = const_cast<void *>(L);   // read only: the digit kernel takes B from LD
        pd.Yout = w.work;
        pd.colexpY = a->cy;
        cudaMemcpyAsync(a->d_tcdesc, &pd, sizeof(pd), cudaMemcpyHostToDevice, st);
        // the row products: G = A_C = L_C D L_KK^T, Abar_C = Lbar_C D^{-1} M
        ProbDesc base = make_desc(p, w, SELINV_F64, L, D, a->Ab, false);
        base.linvd = a->sd;
        base.linvd_off = a->d_sd_off;
        base.linvexp = a->sdexp;
        ProbDesc pdp[2] = {base, base};
        pdp[0].L = L; pdp[0].LD = w.work; pdp[0].prod_op = 0;
        pdp[1].L = a->Lbw; pdp[1].LD = a->Ab; pdp[1].prod_op = 0;
        cudaMemcpyAsync(a->d_pdp + 3, pdp, sizeof(pdp), cudaMemcpyHostToDevice, st);
        launch_lhat_digits(a->d_tcdesc, a->d_dig, (int)a->dig_work.size(), st);
        note_launch();
    }
    const int nl = p.nlevels;
    auto levels = [&](cudaStream_t st) {
        for (int li = nl - 1; li >= 0; li--) {  // root level first
            const int d0 = (int)a->dig_lptr[li], d1 = (int)a->dig_lptr[li + 1];
            if (d1 > d0)
                for (int e : a->tc_launch[li]) {
                    launch_with(a->tcs, a->tcs.launches[e], a->d_tcdesc, st);
                    note_launch();
                }
            for (int b = 0; b < kNumBuckets; b++) {
                const int b0 = a->sm_bptr[li * kNumBuckets + b], b1 = a->sm_bptr[li * kNumBuckets + b + 1];
                launch_bucket(1, b, a->d_desc, a->d_sm + b0, b1 - b0, st);
            }
            const int w0 = (int)a->wd_lptr[li], w1 = (int)a->wd_lptr[li + 1];
            if (w1 > w0) { k_fadj_pull_tc<<<w1 - w0, 256, 0, st>>>(a->d_desc, a->d_wd + w0, w1 - w0); note_launch(); }
            for (int b = 0; b < kNumBuckets; b++) {
                const int b0 = a->sm_bptr[li * kNumBuckets + b], b1 = a->sm_bptr[li * kNumBuckets + b + 1];
                launch_bucket(2, b, a->d_desc, a->d_sm + b0, b1 - b0, st);
            }
            const int m0 = (int)a->mbp_lptr[li], m1 = (int)a->mbp_lptr[li + 1];
            row_product<RP_FAC>(a, 3, li, st);
            if (m1 > m0) {
                k_adj_rowprod<RP_FNBP><<<m1 - m0, kThreads, 0, st>>>(a->d_desc, a->d_mbp + m0, m1 - m0);
                note_launch();
            }
            row_product<RP_FABAR>(a, 4, li, st);
            const int64_t c0 = a->c_lptr[li], c1 = a->c_lptr[li + 1];
            const int64_t j0 = a->j_lptr[li], j1 = a->j_lptr[li + 1];
            if (c1 > c0) { k_fadj_nbar<<<(int)(c1 - c0), 256, 0, st>>>(a->d_desc, a->d_citems + c0, (int)(c1 - c0)); note_launch(); }
            launch_level_gemm(a, OP_FAC_T2, li, st);
            launch_level_gemm(a, OP_FAC_U, li, st);
            if (j1 > j0) {
                k_fadj_ubar<<<dim3((int)(j1 - j0), kFinY), 256, 0, st>>>(a->d_desc, a->d_js + j0, (int)(j1 - j0));
                note_launch();
            }
            launch_level_gemm(a, OP_FAC_T3, li, st);
            launch_level_gemm(a, OP_FAC_G1, li, st);
            launch_level_gemm(a, OP_FAC_G2, li, st);
            if (j1 > j0) {
                k_fadj_fold<<<dim3((int)(j1 - j0), kFinY), 256, 0, st>>>(a->d_desc, a->d_js + j0, (int)(j1 - j0));
                note_launch();
                const int z0 = (int)a->cz_lptr[li], z1 = (int)a->cz_lptr[li + 1];
                if (tc && li > 0 && z1 > z0) {
                    k_adj_colexpz<<<z1 - z0, 256, 0, st>>>(a->d_desc, a->Ab, w.colexpZ, a->d_cz + z0, z1 - z0);
                    note_launch();
                }
            }
        }
    };
    if ((rc = run_captured(a->g_fac, a->g_fac_n, a->g_fac_key, a->g_fac_ws, a->gen, w.colexpZ, st, levels))) return rc;
    if (f->nnzA > 0) {
        const int blocks = (int)std::min<int64_t>((f->nnzA + 255) / 256, 152 * 8);
        k_gather_vals<<<blocks, 256, 0, st>>>(f->d_a_pos, a->Ab, f->nnzA, static_cast<double *>(Abar_vals));
        note_launch();
    }
    return cudaGetLastError() == cudaSuccess ? SELINV_OK : SELINV_ERR_CUDA;
}
