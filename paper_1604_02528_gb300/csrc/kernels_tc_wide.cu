// A^{-1}_{C,K} = -A^{-1}_{C,C} Lhat_{C,K} (Alg. 1, the product after the
// gather) on tcgen05 for supernodes wider than 64 columns, in the transposed
// orientation: the MMA's 128 rows (tensor-memory lanes) are the columns of
// K and its N dimension runs over 64 rows of C, so that every gathered
// entry of A^{-1}_{C,C} is cut into digits once for all of K's columns
// (the row-tile orientation of k_selinv_tc covers at most 64 columns per
// CTA and would gather and slice each entry once per 64 columns).
//
//   A = Lhat^T digit planes: rows = the s columns of K (zero past s), k = the
//       rows q of C; already stored in this operand layout (one contiguous
//       block of roundup(s, 64) x 16 per plane and 16-q step), brought in by
//       bulk copies;
//   B = A^{-1}_{C,C} digit planes: rows = 64 rows p of C, k = q; 8 producer
//       warps gather the entries and slice them with integer operations;
//   D (tensor memory) = 7 group accumulators of 128 x 64, group g holding
//       the exact fp32 sum of the digit products with i + j = g;
//   every 128 k the groups are read back (tcgen05.ld) by 8 epilogue warps
//   and their exact sum is added into a 96-bit word per entry in shared
//   memory (an int64 high part and a 32-bit low part, carried after every
//   chunk).
// Operand rings: 3 stages for the Lhat^T copies, 3 for the gathered digits.
// The copies are issued by a thread of their own, so that the thread issuing
// the products never waits for products to finish: it waits only for its
// operands, and the tensor cores always have the next step queued.
// The same digit scheme and exponent grids as k_selinv_tc; the chunk
// boundaries sit at fixed multiples of 128 k, so the result does not depend
// on the k-split.
//
// Complex symmetric values (template CPLX) run the same contraction on the
// real 2c-long k dimension k' = 2q + part: B(p, 2q) = Re A^{-1}(p, q),
// B(p, 2q + 1) = Im A^{-1}(p, q), and the 2s rows of A are
// [Re Lhat, -Im Lhat] (rows j: the real part of column j of the product)
// and [Im Lhat, Re Lhat] (rows s + j: its imaginary part), so one real
// contraction holds the four real products of the complex one.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "fixedpoint.cuh"
#include "launch.h"
#include "tc_digits.cuh"
#include "tile_gemm.cuh"
#include "umma.cuh"

namespace selinv {

constexpr int kTwN = 64;           // rows of C per item: N of one digit plane
constexpr int kTwProd = 8;         // producer warps: 64 rows x 4 quarters of a 16-k step, 4 values per thread
constexpr int kTwEpi = 8;          // epilogue warps: two per tensor-memory lane quarter (32 rows of C each)
constexpr int kTwMmaWarp = kTwProd + kTwEpi;   // one thread issues the products
constexpr int kTwCopyWarp = kTwMmaWarp + 1;     // one thread issues the Lhat^T copies
constexpr int kTwThreads = 32 * (kTwProd + kTwEpi + 2);
constexpr int kTwHS = kTcM + 1;    // words per row of C in the int64 sums [p][m]: conflict-free both ways
constexpr int kTwAS = 3;           // stages of the Lhat^T ring
constexpr int kTwBS = 3;           // stages of the gathered-digit ring
constexpr int kTwPrefetch = 8;     // steps ahead at which the Lhat^T blocks are asked into L2
static_assert(2 * kTcM * kTwN + kTwN / 2 <= kTcSlotWords, "a split-k slot holds the (hi, lo) words and rowE");

struct TwCfg {
    static constexpr int A_PLANE = kTcM * 16;    // fp16 elements of one Lhat^T digit plane per k16 step
    static constexpr int B_PLANE = kTwN * 16;    // ... of one gathered digit plane
    static constexpr int A_STAGE = kTcDig * A_PLANE;
    static constexpr int B_STAGE = kTcDig * B_PLANE;
    static constexpr uint32_t TCOLS = 512;       // 7 groups x 64 columns
    static constexpr size_t SMEM = sizeof(uint16_t) * (size_t)(kTwAS * A_STAGE + kTwBS * B_STAGE) +
                                   (sizeof(long long) + sizeof(uint32_t)) * (size_t)kTwN * kTwHS + sizeof(int) * kTwN;
};
static_assert(TwCfg::SMEM + 2048 <= 232448, "dynamic + static shared memory within the opt-in limit");

// One chunk's group sums (g weighted 256^(6 - g)), exact, added into the
// entry's 96-bit sum hi 2^32 + lo (0 <= lo < 2^32): the chunk's value is
// h 2^32 + l with h = g0 2^16 + g1 2^8 + g2 and l = g3 2^24 + g4 2^16 +
// g5 2^8 + g6 (|l| < 2^48), and what lo cannot hold is carried into hi.
// Groups 0 and 1 (one and two digit pairs: |g| <= 2^22) are converted by the
// exact magic-number addition on the FP32 pipe, the others by F2I, whose
// unit is the epilogue's bottleneck.
__device__ __forceinline__ void add_chunk(const uint32_t (&acc)[kTcDig][8], int jj, bool first, long long &hi,
                                          uint32_t &lo) {
    long long gv[kTcDig];
#pragma unroll
    for (int gq = 0; gq < 2; gq++)
        gv[gq] = (long long)(__float_as_int(__fadd_rn(__uint_as_float(acc[gq][jj]), 12582912.0f)) - 0x4B400000);
#pragma unroll
    for (int gq = 2; gq < kTcDig; gq++) gv[gq] = (long long)__float2int_rn(__uint_as_float(acc[gq][jj]));
    const long long h = (gv[0] << 16) + (gv[1] << 8) + gv[2];
    const long long l = (gv[3] << 24) + (gv[4] << 16) + (gv[5] << 8) + gv[6];
    const long long t = (first ? 0ll : (long long)lo) + l;
    hi = (first ? 0ll : hi) + h + (t >> 32);
    lo = (uint32_t)t;
}

// items: tile = (row tile * nmt + m tile) * nsplit + k-range, ntiles = nsplit;
// nmt = ceil(rows of A / 128) (1 for real supernodes of <= 128 columns).
//
// SYRK: the update that the reverse pass of the gather hands to the
// ancestors, V_K -= [Ybar, Lhat] [Lhat, Ybar]^T over the 2s columns (lower
// triangle of the c x c update matrix, its diagonal halved): A = digit
// planes of [Ybar, Lhat] for 128 rows of C (k_syrk_digits, one exponent per
// row), B = 64 rows of [Lhat, Ybar] sliced here; items (K, 128-row block *
// number of 64-row blocks + 64-row block) on or below the diagonal.
//
// LHAT: the same machinery forms products of a panel's rows with an s x s
// matrix, out(p, j) = sum_k X(p, k) B(k, j) for the rows p of C: A = digit
// planes of B transposed (rows = the columns j, k = the s columns of the
// panel, in this operand layout, with an exponent per column j), B = 64
// rows of the dense panel X (row exponent over the row's s entries), k = s:
// a single chunk, no k-split.  The forward's Lhat_{C,K} = L_{C,K} L_KK^{-1}
// (Alg. 1, first loop; digits by k_linv_digits) goes to Lhat's slots of the
// LD panel; the reverse passes' row products use the other prod_op modes.
template <bool CPLX, bool LHAT = false, bool SYRK = false>
__global__ void __launch_bounds__(kTwThreads, 1) k_selinv_tcw(const ProbDesc *__restrict__ descs,
                                                              const Item *__restrict__ items, int nitems,
                                                              long long *__restrict__ slab, long long wait_limit) {
    grid_dep_wait();
    using Cfg = TwCfg;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);                    // [kTwAS][7][A_PLANE] Lhat^T digits
    uint16_t *Bs = As + kTwAS * Cfg::A_STAGE;                                  // [kTwBS][7][B_PLANE] gathered digits
    long long *Hi = reinterpret_cast<long long *>(Bs + kTwBS * Cfg::B_STAGE);  // [64 p][kTwHS] high words of the sums
    uint32_t *Lo = reinterpret_cast<uint32_t *>(Hi + kTwN * kTwHS);          // [64 p][kTwHS] low 32 bits
    int *rowE = reinterpret_cast<int *>(Lo + kTwN * kTwHS);                   // [64]
    __shared__ int64_t tile_cb[kTwN], tile_rb[kTwN];
    // full[s] / bempty[s]: the producers wrote B of stage s / the products
    // that read it are done; afull[s] / aempty[s]: the bulk copies of A landed
    // in stage s / the products that read it are done; acc_full: a chunk's
    // group sums are complete; tmem_free: the epilogue read them; drain:
    // every product issued before an abort is done
    __shared__ __align__(8) uint64_t full[kTwBS], bempty[kTwBS], afull[kTwAS], aempty[kTwAS], acc_full, tmem_free,
        drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_pre;
    __shared__ volatile int s_abort;
    __shared__ int ymax[kTcM];

    const int w = blockIdx.x;
    if (w >= nitems) return;
    const long long mlim = wait_limit > kMbarMinPolls ? wait_limit : kMbarMinPolls;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const Item it = items[w];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    constexpr bool DENSE = LHAT || SYRK;                 // B from dense panels
    const int kw = SYRK ? 2 * s : (LHAT ? s : (CPLX ? 2 * c : c));   // k extent
    const int mrows = SYRK ? c : (CPLX ? 2 * s : s);     // rows of A (output rows)
    // operand rows of a stored digit block (SYRK: blocks of exactly 128 rows)
    const int s64 = SYRK ? kTcM : (mrows + 63) / 64 * 64;
    const int nmt = SYRK ? 1 : (mrows + kTcM - 1) / kTcM;
    const int nsplit = it.ntiles;
    const int ksp = it.tile % nsplit;
    const int n2 = (c + kTwN - 1) / kTwN;                // SYRK: 64-row blocks of C
    const int mt = SYRK ? 0 : (it.tile / nsplit) % nmt;
    const int tile = SYRK ? it.tile % n2 : it.tile / nsplit / nmt;
    const int p0 = tile * kTwN, m0 = SYRK ? (it.tile / n2) * kTcM : mt * kTcM;
    const int64_t pos0 = P.rowptr[K] + s;
    const int nsteps = (kw + 15) / 16;
    const int chunk = ((nsteps + nsplit - 1) / nsplit + kTcFlush - 1) / kTcFlush * kTcFlush;
    const int st0 = ksp * chunk;
    const int st1 = st0 + chunk < nsteps ? st0 + chunk : nsteps;
    const int n = st1 > st0 ? st1 - st0 : 0;             // k16 steps of this item
    const int nflush = (n + kTcFlush - 1) / kTcFlush;
    const int arows = SYRK ? kTcM : (s64 - m0 < kTcM ? s64 - m0 : kTcM);   // rows of A in the stored blocks

    int a_issued = -1;   // last step whose A copies the MMA thread issued
    // copies of the Lhat^T digit planes of step i_ (rows m0 .. m0 + 127 of
    // each stored block); the 7 planes of a step lie one after the other, so
    // a block of exactly 128 rows comes in one copy
    const uint16_t *Au = SYRK ? P.linvd + P.linvd_off[K] + (int64_t)(m0 / kTcM) * nsteps * kTcDig * kTcM * 16
                              : (LHAT ? P.linvd + P.linvd_off[K] : P.lhsu + P.lhsu_off[K]) + (int64_t)(m0 / 8) * 128;
    const uint32_t aBytes = (uint32_t)(arows * 16 * 2);
    const bool whole = SYRK || (m0 == 0 && s64 == kTcM);
    auto load_a = [&](int i_) {
        const int st = i_ % kTwAS;
        const uint16_t *src = Au + (int64_t)(st0 + i_) * kTcDig * s64 * 16;
        umma::mbar_arrive_expect_tx(&afull[st], kTcDig * aBytes);
        if (whole) {
            umma::bulk_g2s(As + st * Cfg::A_STAGE, src, kTcDig * aBytes, &afull[st]);
        } else {
#pragma unroll
            for (int pl = 0; pl < kTcDig; pl++)
                umma::bulk_g2s(As + st * Cfg::A_STAGE + pl * Cfg::A_PLANE, src + (int64_t)pl * s64 * 16, aBytes,
                               &afull[st]);
        }
        a_issued = i_;
    };
    if (tid == 0) {
        s_pre = 0;
        s_abort = 0;
        for (int st = 0; st < kTwBS; st++) {
            umma::mbar_init(&full[st], kTwProd);
            umma::mbar_init(&bempty[st], 1);
        }
        for (int st = 0; st < kTwAS; st++) {
            umma::mbar_init(&afull[st], 1);      // the arrival that expects A's bytes
            umma::mbar_init(&aempty[st], 1);
        }
        umma::mbar_init(&acc_full, 1);
        umma::mbar_init(&tmem_free, kTwEpi);
        umma::mbar_init(&drain, 1);
        umma::mbar_init_fence();
    }
    // rows of A past the stored blocks stay zero in every stage (the copies
    // write only the rows before them)
    if (arows < kTcM)
        for (int st = 0; st < kTwAS; st++)
            for (int pl = 0; pl < kTcDig; pl++)
                for (int e = arows * 16 + tid * 8; e < Cfg::A_PLANE; e += kTwThreads * 8)
                    *reinterpret_cast<uint4 *>(As + st * Cfg::A_STAGE + pl * Cfg::A_PLANE + e) = make_uint4(0, 0, 0, 0);
    if (DENSE)
        for (int e = tid; e < kTwN; e += kTwThreads) rowE[e] = 0;
    umma::fence_proxy_async();   // zeroed A rows are seen by the tensor cores
    __syncthreads();
    // the first copies (one per stage) go out before the rest of the set-up;
    // the blocks of the steps after them are asked into L2 (the CTAs of one
    // supernode run in step, so each block would otherwise come from DRAM for
    // all of them)
    if (warp == kTwCopyWarp && lane == 0) {
        for (int i_ = 0; i_ < kTwAS && i_ < n; i_++) load_a(i_);
        for (int i_ = kTwAS; i_ < kTwPrefetch && i_ < n; i_++)
            umma::bulk_prefetch_l2(Au + (int64_t)(st0 + i_) * kTcDig * s64 * 16, kTcDig * aBytes);
    }
    if constexpr (DENSE) {
        // row exponents of the dense B rows: row p over its kw entries (LHAT:
        // the panel L; SYRK: [Lhat, Ybar] from the panels L and Z)
        const int r = tid % kTwN;
        int e = 0;
        if (p0 + r < c)
            for (int k = tid / kTwN; k < kw; k += kTwThreads / kTwN) {
                const double *src = static_cast<const double *>(SYRK && k >= s ? P.Z : P.L);
                e = max(e, bexp(src[P.panel_off[K] + (int64_t)(SYRK && k >= s ? k - s : k) * ld + s + p0 + r]));
            }
        if (e) atomicMax(&rowE[r], e);
    } else {
        // row exponents of the gathered block: row p is bounded by the largest
        // whole-column exponent of A^{-1} over C[0..p] (entry (p, q) sits in
        // the ancestor column C[min(p, q)])
        int e = 0;
        for (int q = tid; q < p0 && q < c; q += kTwThreads) e = max(e, P.colexpZ[P.rows[pos0 + q]]);
        if (e) atomicMax(&s_pre, e);
        for (int i = tid; i < kTwN; i += kTwThreads) {
            const int p = p0 + i;
            tile_cb[i] = p < c ? P.colbase[pos0 + p] : 0;
            tile_rb[i] = p < c ? P.relbase[pos0 + p] : 0;
            rowE[i] = p < c ? P.colexpZ[P.rows[pos0 + p]] : 0;
        }
    }
    // the sums are written by the first flush; an item without steps leaves zeros
    if (n == 0)
        for (int e = tid; e < kTwN * kTwHS; e += kTwThreads) {
            Hi[e] = 0;
            Lo[e] = 0;
        }
    for (int e = tid; e < kTcM; e += kTwThreads) ymax[e] = 0;
    if (warp == kTwMmaWarp) {
        umma::tmem_alloc(&s_tmem, Cfg::TCOLS);
        umma::tmem_relinquish();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (!DENSE && warp == 0) {   // prefix max over the 64 rows
        int carry = s_pre;
        for (int b = 0; b < kTwN; b += 32) {
            int v = max(rowE[b + lane], carry);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = max(v, u);
            }
            rowE[b + lane] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    const uint32_t tmem = s_tmem;

    if (warp < kTwProd) {
        // ---- producers: thread (row r, quarter kq) slices the k-values
        // 4 kq .. 4 kq + 3 of each 16-k step; a warp holds 16 rows x 2
        // quarters, so that its stores of a plane fill two 128-byte core
        // matrices.  Complex: the 4 k-values are (Re, Im) of the entries
        // q = 8 step + 2 kq and + 1.  The gather runs three steps ahead in
        // registers, every load a whole step before its use: column data
        // (step i + 3), relative rows (i + 2), values (i + 1).
        const TcGather g{P.colbase + pos0, P.relbase + pos0, P.relidx, tile_cb, tile_rb, p0, c, gather_check(P)};
        const int r = (warp % 4) * 16 + (lane >> 1), kq = (warp / 4) * 2 + (lane & 1);
        const int E = rowE[r];
        constexpr int NV = CPLX ? 2 : 4;        // entries of A^{-1}_{C,C} per thread and step
        constexpr int QS = CPLX ? 8 : 16;       // entries per step
        double v[4];
        int64_t ab[NV], cb[NV], rb[NV];
        int32_t ar[NV];
        bool up[NV];
        // Hermitian: an entry above the diagonal is the conjugate of the stored one
        const bool herm = CPLX && P.herm;
        auto load = [&]() {
            if (CPLX) {
                const double2 *Zc = static_cast<const double2 *>(P.Z);
#pragma unroll
                for (int u = 0; u < NV; u++) {
                    const double2 z = ab[u] >= 0 ? Zc[ab[u] + ar[u]] : make_double2(0.0, 0.0);
                    v[2 * u] = z.x;
                    v[2 * u + 1] = herm && up[u] ? -z.y : z.y;
                }
            } else {
                const double *Zg = static_cast<const double *>(P.Z);
#pragma unroll
                for (int u = 0; u < NV; u++) v[u] = ab[u] >= 0 ? Zg[ab[u] + ar[u]] : 0.0;
            }
        };
        // column data of step i_ (of this item), none past the last step
        auto cols = [&](int i_) {
#pragma unroll
            for (int u = 0; u < NV; u++) {
                if (i_ < n) g.cols((st0 + i_) * QS + kq * NV + u, cb[u], rb[u]);
                else { cb[u] = -1; rb[u] = 0; }
            }
        };
        // DENSE: the 4 values of step i_ straight from the dense panel(s)
        const double *Lc = static_cast<const double *>(P.L) + P.panel_off[K] + s + p0 + r;   // X(p0 + r, k) = Lc[k ld]
        const double *Zc2 = static_cast<const double *>(P.Z) + P.panel_off[K] + s + p0 + r;  // SYRK: k >= s
        const bool rok = p0 + r < c;
        auto load_dense = [&](int i_) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int k = (st0 + i_) * 16 + kq * 4 + u;
                v[u] = (rok && i_ < n && k < kw) ? (SYRK && k >= s ? Zc2[(int64_t)(k - s) * ld] : Lc[(int64_t)k * ld]) : 0.0;
            }
        };
        auto parts = [&](int i_) {
#pragma unroll
            for (int u = 0; u < NV; u++) {
                if (i_ < n) g.parts(r, (st0 + i_) * QS + kq * NV + u, cb[u], rb[u], ab[u], ar[u], up[u]);
                else { ab[u] = -1; ar[u] = 0; }
            }
            // bounds check (debug): an address outside the panels is dropped
            if (g.chk.on)
#pragma unroll
                for (int u = 0; u < NV; u++)
                    if (ab[u] >= 0 && !g.chk.ok(ab[u] + ar[u])) ab[u] = -1;
        };
        if (DENSE) {
            if (n > 0) load_dense(0);
        } else if (n > 0) {
            cols(0);
            parts(0);
            load();
            cols(1);
            parts(1);
            cols(2);
        }
        for (int i_ = 0; i_ < n; i_++) {
            const int stage = i_ % kTwBS, use = i_ / kTwBS;
            uint16_t *Bb = Bs + stage * Cfg::B_STAGE;
            if (i_ >= kTwBS && !umma::mbar_wait(&bempty[stage], (uint32_t)((use - 1) & 1), mlim)) {
                s_abort = 1;
                break;
            }
            {
                uint32_t lo[4], hi[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const unsigned long long wv = (unsigned long long)(fixed54(v[u], E) + 0x80808080808080ll);
                    lo[u] = (uint32_t)wv;
                    hi[u] = (uint32_t)(wv >> 32);
                }
                uint16_t *dst = Bb + (r / 8) * 128 + (kq / 2) * 64 + (r % 8) * 8 + (kq % 2) * 4;
                store_plane4<0>(dst + 0 * Cfg::B_PLANE, lo, hi);
                store_plane4<1>(dst + 1 * Cfg::B_PLANE, lo, hi);
                store_plane4<2>(dst + 2 * Cfg::B_PLANE, lo, hi);
                store_plane4<3>(dst + 3 * Cfg::B_PLANE, lo, hi);
                store_plane4<4>(dst + 4 * Cfg::B_PLANE, lo, hi);
                store_plane4<5>(dst + 5 * Cfg::B_PLANE, lo, hi);
                store_plane4<6>(dst + 6 * Cfg::B_PLANE, lo, hi);
            }
            // release the step's operand first: the loads of later steps are
            // issued after the arrival, not between the stores and the fence
            umma::fence_proxy_async();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&full[stage]);
            if (DENSE) {
                load_dense(i_ + 1);
            } else {
                load();            // values of step i + 1
                parts(i_ + 2);     // relative rows of step i + 2
                cols(i_ + 3);      // column data of step i + 3
            }
            if (s_abort) break;
        }
    } else if (warp == kTwMmaWarp) {
        // ---- one thread issues the products once both operands of a step
        // have landed (and, at the start of a chunk, the epilogue has read the
        // group sums of the previous one)
        if (lane == 0) {
            for (int i_ = 0; i_ < n; i_++) {
                const int sa = i_ % kTwAS, sb = i_ % kTwBS, ch = i_ / kTcFlush;
                const bool first = i_ % kTcFlush == 0;
                if (!umma::mbar_wait(&afull[sa], (uint32_t)((i_ / kTwAS) & 1), mlim) ||
                    !umma::mbar_wait(&full[sb], (uint32_t)((i_ / kTwBS) & 1), mlim) ||
                    (first && ch > 0 && !umma::mbar_wait(&tmem_free, (uint32_t)((ch - 1) & 1), mlim))) {
                    s_abort = 1;
                    break;
                }
                umma::fence_after_sync();
                const uint64_t ad0 = umma::smem_desc(umma::smem_u32(As + sa * Cfg::A_STAGE), 128, 256);
                const uint64_t bd0 = umma::smem_desc(umma::smem_u32(Bs + sb * Cfg::B_STAGE), 128, 256);
                digit_products<kTwN, Cfg::A_PLANE, Cfg::B_PLANE>(tmem, ad0, bd0, first);
                umma::commit(&aempty[sa]);
                umma::commit(&bempty[sb]);
                if (i_ % kTcFlush == kTcFlush - 1 || i_ == n - 1) umma::commit(&acc_full);
                if (s_abort) break;
            }
        }
        __syncwarp();
    } else if (warp == kTwCopyWarp) {
        // ---- one thread copies the Lhat^T digit planes of step i into the
        // stage of step i - 3 once the products of that step are done (the
        // first three went out during the set-up)
        if (lane == 0) {
            for (int i_ = kTwAS; i_ < n; i_++) {
                if (!umma::mbar_wait(&aempty[i_ % kTwAS], (uint32_t)((i_ / kTwAS - 1) & 1), mlim)) {
                    s_abort = 1;
                    break;
                }
                load_a(i_);
                if (i_ + kTwPrefetch - kTwAS < n)
                    umma::bulk_prefetch_l2(Au + (int64_t)(st0 + i_ + kTwPrefetch - kTwAS) * kTcDig * s64 * 16,
                                           kTcDig * aBytes);
                if (s_abort) break;
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: every chunk's exact fp32 group sums -> the 96-bit sums;
        // warp (lane quarter, half) reads output rows 32 (warp % 4) .. + 31
        // and rows of C 32 half .. + 31
        const int lb = 32 * (warp % 4), m = lb + lane, half = (warp / 4) & 1;
        for (int f = 0; f < nflush; f++) {
            if (!umma::mbar_wait(&acc_full, (uint32_t)(f & 1), mlim)) {
                s_abort = 1;
                break;
            }
            umma::fence_after_sync();
#pragma unroll 1
            for (int cb = 0; cb < 4; cb++) {
                uint32_t acc[kTcDig][8];
#pragma unroll
                for (int gq = 0; gq < kTcDig; gq++)
                    umma::tmem_ld8(tmem + ((uint32_t)lb << 16) + (uint32_t)(gq * kTwN + half * 32 + cb * 8), acc[gq]);
                umma::tmem_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {   // the first chunk writes, the later ones add
                    const int e = (half * 32 + cb * 8 + jj) * kTwHS + m;
                    add_chunk(acc, jj, f == 0, Hi[e], Lo[e]);
                }
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&tmem_free);
            if (s_abort) break;
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (s_abort) {
        // a wait ran out: report, wait (bounded) for the products this CTA
        // issued (a commit after the last of them) and for its last bulk
        // copies, release the tensor memory and leave
        if (tid == 0) atomicCAS(P.status, 0, SELINV_ERR_TIMEOUT);
        if (warp == kTwMmaWarp && lane == 0) {
            umma::commit(&drain);
            umma::mbar_wait(&drain, 0u, mlim);
        }
        if (warp == kTwCopyWarp && lane == 0)   // the copies that may still be in flight
            for (int j = a_issued - (kTwAS - 1) > 0 ? a_issued - (kTwAS - 1) : 0; j <= a_issued; j++)
                umma::mbar_wait(&afull[j % kTwAS], (uint32_t)((j / kTwAS) & 1), mlim);
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (warp == kTwMmaWarp) umma::tmem_dealloc(tmem, Cfg::TCOLS);
        return;
    }
    umma::fence_after_sync();
    if (warp == kTwMmaWarp) umma::tmem_dealloc(tmem, Cfg::TCOLS);

    // Y = -(A^{-1}_{C,C} Lhat): B digits on 2^(E - 1028 - 8i) of the row of
    // C, A digits on 2^(F - 1029 - 8j) of the column of K, so the value is
    // (hi 2^-16 + lo 2^-48) 2^(E + F - 2057); LHAT: Lhat = L_{C,K} L_KK^{-1}
    // on the same grids (F: the column exponent of L_KK^{-1})
    if constexpr (SYRK) {
        // V_K(p1, p2) -= the product, p1 >= p2, the diagonal halved (exactly:
        // one less in the scale); A's rows carry their own exponents
        double *V = static_cast<double *>(P.Yout) + P.part_off[K];
        for (int e = tid; e < kTwN * kTcM; e += kTwThreads) {
            const int p = e % kTwN, mm = e / kTwN, p1 = m0 + mm, p2 = p0 + p;
            if (p1 >= c || p2 >= c || p1 < p2) continue;
            const int sc = (rowE[p] - 1022) + (P.linvexp[pos0 + p1] - 1022) - 13 - (p1 == p2 ? 1 : 0);
            V[(int64_t)p2 * c + p1] -= fixed_to_double(Hi[p * kTwHS + mm], (long long)Lo[p * kTwHS + mm], sc);
        }
        return;
    }
    if constexpr (LHAT) {
        double *Lh = static_cast<double *>(P.LD) + P.panel_off[K];
        const double *Ad = static_cast<const double *>(P.Yout) + P.panel_off[K];
        const int op = P.prod_op;
        for (int e = tid; e < kTwN * kTcM; e += kTwThreads) {
            const int p = e % kTwN, j = e / kTwN;
            if (p0 + p >= c || j >= s) continue;
            const int sc = (rowE[p] - 1022) + (P.linvexp[fc + j] - 1022) - 13;
            const double y = fixed_to_double(Hi[p * kTwHS + j], (long long)Lo[p * kTwHS + j], sc);
            const int64_t at = (int64_t)j * ld + s + p0 + p;
            if (op == 0) Lh[at] = y;
            else if (op == 1) Lh[at] -= y;
            else Lh[at] = Ad[at] - y;
        }
        return;
    }
    if (nsplit == 1) {
        double *Zk = static_cast<double *>(P.Yout) + (CPLX ? 2 : 1) * P.panel_off[K];
        for (int e = tid; e < kTwN * kTcM; e += kTwThreads) {
            const int p = e % kTwN, mm = e / kTwN, jr = m0 + mm;   // a warp shares mm
            if (p0 + p >= c || jr >= mrows) continue;
            const int j = CPLX && jr >= s ? jr - s : jr;
            const int sc = (rowE[p] - 1022) + (P.colexp[fc + j] - 1022) - 13;
            const double y = fixed_to_double(Hi[p * kTwHS + mm], (long long)Lo[p * kTwHS + mm], sc);
            const int64_t at = (int64_t)j * ld + s + p0 + p;
            if (CPLX) Zk[2 * at + (jr >= s ? 1 : 0)] = -y;
            else Zk[at] = -y;
            warp_uniform_atomic_max(&ymax[mm], bexp(y));
        }
    } else {
        // split k: the partial tile and the rows' exponents go to this CTA's
        // slab slot, [output row][row of C]; k_tcw_reduce sums the slots
        long long *mine = slab + (int64_t)blockIdx.x * kTcSlotWords;
        for (int e = tid; e < kTwN * kTcM; e += kTwThreads) {
            const int p = e % kTwN, mm = e / kTwN;
            mine[e] = Hi[p * kTwHS + mm];
            mine[kTwN * kTcM + e] = (long long)Lo[p * kTwHS + mm];
        }
        int *re = reinterpret_cast<int *>(mine + 2 * kTwN * kTcM);
        for (int e = tid; e < kTwN; e += kTwThreads) re[e] = rowE[e];
        return;
    }
    __syncthreads();
    // column exponents of A^{-1}_{C,K} over all row tiles (used by the diagonal block)
    for (int mm = tid; mm < kTcM; mm += kTwThreads) {
        const int jr = m0 + mm;
        if (jr < mrows && ymax[mm] > 0) atomicMax(&P.colexpY[fc + (CPLX && jr >= s ? jr - s : jr)], ymax[mm]);
    }
}

// Split-k reduction of k_selinv_tcw: one CTA per (row tile of 64, 8 output
// rows); each element adds the (hi, lo) words of the group's k-range slots
// (exact integer sums) and forms A^{-1}_{C,K} = -(sum).
// red[w] = {index of the group's first item, its slab slot, block of 8 output rows}.
template <bool CPLX>
__global__ void __launch_bounds__(256) k_tcw_reduce(const ProbDesc *__restrict__ descs,
                                                    const Item *__restrict__ items, const int4 *__restrict__ red,
                                                    int nred, const long long *__restrict__ slab) {
    grid_dep_wait();
    __shared__ int ymax[8];
    const int w = blockIdx.x;
    if (w >= nred) return;
    const int4 rr = red[w];
    const Item it = items[rr.x];
    const ProbDesc &P = descs[it.prob];
    const int K = it.K;
    const int fc = P.super_ptr[K];
    const int s = P.super_ptr[K + 1] - fc;
    const int64_t ld = P.rowptr[K + 1] - P.rowptr[K];
    const int c = (int)(ld - s);
    const int mrows = CPLX ? 2 * s : s;
    const int nmt = (mrows + kTcM - 1) / kTcM;
    const int nsplit = it.ntiles;
    const int mt = (it.tile / nsplit) % nmt;
    const int p0 = (it.tile / nsplit / nmt) * kTwN, m0 = mt * kTcM;
    const int *rowE = reinterpret_cast<const int *>(slab + (int64_t)rr.y * kTcSlotWords + 2 * kTwN * kTcM);
    if (threadIdx.x < 8) ymax[threadIdx.x] = 0;
    __syncthreads();
    double *Zk = static_cast<double *>(P.Yout) + (CPLX ? 2 : 1) * P.panel_off[K];
    const int p = threadIdx.x % kTwN;
    for (int r8 = threadIdx.x / kTwN; r8 < 8; r8 += 256 / kTwN) {   // a warp shares r8
        const int mm = rr.z * 8 + r8, jr = m0 + mm;
        if (jr >= mrows || p0 + p >= c) continue;
        long long hi = 0, lo = 0;
        for (int k2 = 0; k2 < nsplit; k2++) {
            const long long *sl = slab + ((int64_t)rr.y + k2) * kTcSlotWords;
            hi += sl[mm * kTwN + p];
            lo += sl[kTwN * kTcM + mm * kTwN + p];
        }
        const int j = CPLX && jr >= s ? jr - s : jr;
        const int sc = (rowE[p] - 1022) + (P.colexp[fc + j] - 1022) - 13;
        const double y = fixed_to_double(hi, lo, sc);
        const int64_t at = (int64_t)j * ld + s + p0 + p;
        if (CPLX) Zk[2 * at + (jr >= s ? 1 : 0)] = -y;
        else Zk[at] = -y;
        warp_uniform_atomic_max(&ymax[r8], bexp(y));
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int jr = m0 + rr.z * 8 + (int)threadIdx.x;
        if (jr < mrows && ymax[threadIdx.x] > 0)
            atomicMax(&P.colexpY[fc + (CPLX && jr >= s ? jr - s : jr)], ymax[threadIdx.x]);
    }
}

cudaError_t configure_tcw_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_selinv_tcw<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TwCfg::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_selinv_tcw<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TwCfg::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_selinv_tcw<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TwCfg::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_selinv_tcw<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TwCfg::SMEM);
    return e;
}

cudaError_t launch_selinv_tcw(int cplx, const ProbDesc *d, const Item *items, int n, long long *slab,
                              long long wait_limit, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (cplx) k_selinv_tcw<true><<<n, kTwThreads, TwCfg::SMEM, st>>>(d, items, n, slab, wait_limit);
    else k_selinv_tcw<false><<<n, kTwThreads, TwCfg::SMEM, st>>>(d, items, n, slab, wait_limit);
    return cudaGetLastError();
}

cudaError_t launch_lhat_tcw(const ProbDesc *d, const Item *items, int n, long long wait_limit, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_selinv_tcw<false, true><<<n, kTwThreads, TwCfg::SMEM, st>>>(d, items, n, nullptr, wait_limit);
    return cudaGetLastError();
}

cudaError_t launch_syrk_tcw(const ProbDesc *d, const Item *items, int n, long long wait_limit, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_selinv_tcw<false, false, true><<<n, kTwThreads, TwCfg::SMEM, st>>>(d, items, n, nullptr, wait_limit);
    return cudaGetLastError();
}

cudaError_t launch_tcw_reduce(int cplx, const ProbDesc *d, const Item *items, const int4 *red, int n,
                              const long long *slab, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (cplx) k_tcw_reduce<true><<<n, 256, 0, st>>>(d, items, red, n, slab);
    else k_tcw_reduce<false><<<n, 256, 0, st>>>(d, items, red, n, slab);
    return cudaGetLastError();
}

}  // namespace selinv
