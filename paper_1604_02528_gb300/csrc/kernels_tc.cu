// A^{-1}_{C,K} = -A^{-1}_{C,C} Lhat_{C,K} (Alg. 1, the product after the
// gather) on the 5th-generation tensor cores: the FP64-exact digit scheme of
// the mma.sync kernel (7 balanced base-256 digits per operand, held in fp16,
// on a row / column exponent grid; digit products grouped by i + j into
// exact fp32 sums, folded into int64 every 128 k), with
//   * a 128-row x TN-column output tile per CTA whose 7 group accumulators
//     live in tensor memory (7 TN columns), written by tcgen05.mma issued from
//     one thread, completion signalled through mbarriers;
//   * operands in shared memory in the K-major layout without swizzle, two
//     stages: while the tensor cores work on step k, 16 producer warps gather
//     the A^{-1}(C,C) entries of step k + 1 and cut them into digits (integer
//     operations only, 4 values per thread), and bulk copies bring the Lhat
//     digit planes of step k + 1;
//   * each MMA takes one A digit plane against up to 256 / TN B planes
//     (digit_products: 10 MMAs per step for TN = 64, 7 for TN <= 32);
//   * every 128 k the group sums are read from tensor memory by 8 epilogue
//     warps and added as int64 into per-element (hi, lo) words in shared
//     memory.
// Split-k items store their int64 words in a per-CTA slab slot; k_tc_reduce,
// launched next, sums the slots of each row tile (exact) and writes A^{-1}_{C,K}.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "fixedpoint.cuh"
#include "launch.h"
#include "tc_digits.cuh"
#include "tile_gemm.cuh"
#include "umma.cuh"

namespace selinv {

constexpr int kTcProd = 16;        // producer warps: gather + digits of A (4 values per thread and step)
constexpr int kTcEpi = 8;          // epilogue warps: two per tensor-memory lane quarter (half the columns each)
constexpr int kTcMmaWarp = kTcProd + kTcEpi;   // one thread issues the products
constexpr int kTcCopyWarp = kTcMmaWarp + 1;     // one thread issues the Lhat digit copies
constexpr int kTcThreads = 32 * (kTcProd + kTcEpi + 2);
// slab slot of a split-k item: (hi, lo) words [64 columns][128 rows] each, then the rows' exponents
constexpr int64_t kTcSlot = kTcSlotWords;
static_assert(kTcSlotWords == 2 * kTcM * 64 + kTcM / 2, "slot layout");
static_assert(kTcProd % 4 == 0, "epilogue warp w reads tensor-memory lanes 32 (w % 4) ..");

template <int TN> struct TcCfg {
    static constexpr int A_PLANE = kTcM * 16;    // bf16 elements of one digit plane per k16 step
    static constexpr int B_PLANE = TN * 16;
    static constexpr int A_STAGE = kTcDig * A_PLANE;
    static constexpr int B_STAGE = kTcDig * B_PLANE;
    static constexpr uint32_t TCOLS = kTcDig * TN <= 128 ? 128u : (kTcDig * TN <= 256 ? 256u : 512u);
    static constexpr size_t SMEM =
        sizeof(uint16_t) * 2 * (size_t)(A_STAGE + B_STAGE) + sizeof(long long) * 2 * (size_t)kTcM * TN +
        sizeof(int) * kTcM;
};

template <int TN>
__global__ void __launch_bounds__(kTcThreads, 1) k_selinv_tc(const ProbDesc *__restrict__ descs,
                                                             const Item *__restrict__ items, int nitems,
                                                             long long *__restrict__ slab, long long wait_limit) {
    grid_dep_wait();
    using Cfg = TcCfg<TN>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);                // [2][7][A_PLANE]
    uint16_t *Bs = As + 2 * Cfg::A_STAGE;                                  // [2][7][B_PLANE]
    long long *Hi = reinterpret_cast<long long *>(Bs + 2 * Cfg::B_STAGE);  // [TN][128]
    long long *Lo = Hi + kTcM * TN;                                        // [TN][128]
    int *rowE = reinterpret_cast<int *>(Lo + kTcM * TN);                   // [128]
    __shared__ int64_t tile_cb[kTcM], tile_rb[kTcM];
    // full[s]: the producer warps wrote A in stage s; bfull[s]: the bulk
    // copies of B landed there; empty[s]: the products that read stage s are
    // done; acc_full: a chunk's group sums are complete in tensor memory;
    // tmem_free: the epilogue warps have read them; drain: every product
    // issued before an abort is done
    __shared__ __align__(8) uint64_t full[2], bfull[2], empty[2], acc_full, tmem_free, drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_pre;
    __shared__ volatile int s_abort;
    __shared__ int ymax[128];

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
    const int c16 = (c + 15) & ~15;
    const int ncol = (s + TN - 1) / TN;
    const int nsplit = it.ntiles;
    const int ksp = it.tile % nsplit;
    const int ct = (it.tile / nsplit) % ncol;
    const int tile = it.tile / nsplit / ncol;
    const int p0 = tile * kTcM, n0 = ct * TN;
    const int64_t pos0 = P.rowptr[K] + s;
    const int nsteps = c16 / 16;
    const int chunk = ((nsteps + nsplit - 1) / nsplit + kTcFlush - 1) / kTcFlush * kTcFlush;
    const int st0 = ksp * chunk;
    const int st1 = st0 + chunk < nsteps ? st0 + chunk : nsteps;
    const int n = st1 > st0 ? st1 - st0 : 0;                 // k16 steps of this item
    const int nflush = (n + kTcFlush - 1) / kTcFlush;

    // row exponents of the gathered block: row p is bounded by the largest
    // whole-column exponent of A^{-1} over C[0..p] (entry (p, q) sits in
    // the ancestor column C[min(p, q)])
    if (tid == 0) { s_pre = 0; s_abort = 0; }
    __syncthreads();
    {
        int e = 0;
        for (int q = tid; q < p0 && q < c; q += kTcThreads) e = max(e, P.colexpZ[P.rows[pos0 + q]]);
        if (e) atomicMax(&s_pre, e);
    }
    for (int e = tid; e < kTcM; e += kTcThreads) {
        const int p = p0 + e;
        tile_cb[e] = p < c ? P.colbase[pos0 + p] : 0;
        tile_rb[e] = p < c ? P.relbase[pos0 + p] : 0;
        rowE[e] = p < c ? P.colexpZ[P.rows[pos0 + p]] : 0;
    }
    // Hi and Lo are written by the first flush; an item without steps leaves zeros
    if (n == 0)
        for (int e = tid; e < 2 * kTcM * TN; e += kTcThreads) Hi[e] = 0;
    for (int e = tid; e < 128; e += kTcThreads) ymax[e] = 0;
    if (tid == 0) {
        for (int st = 0; st < 2; st++) {
            umma::mbar_init(&full[st], kTcProd);
            umma::mbar_init(&bfull[st], 1);     // the arrival that expects B's bytes
            umma::mbar_init(&empty[st], 1);
        }
        umma::mbar_init(&acc_full, 1);
        umma::mbar_init(&tmem_free, kTcEpi);
        umma::mbar_init(&drain, 1);
        umma::mbar_init_fence();
    }
    if (warp == kTcMmaWarp) {
        umma::tmem_alloc(&s_tmem, Cfg::TCOLS);
        umma::tmem_relinquish();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) {                          // prefix max over the 128 rows
        int carry = s_pre;
        for (int b = 0; b < kTcM; b += 32) {
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
    int b_issued = -1;   // last step whose B copies the copy thread issued
    // copies of the Lhat digit planes of step i_ (bulk, tcgen05 layout: one
    // contiguous block per plane and step) into stage i_ % 2
    const int64_t s64 = (s + 63) / 64 * 64;
    const uint16_t *Bu = P.lhsu + P.lhsu_off[K] + (int64_t)(n0 / 8) * 128;
    constexpr uint32_t kBBytes = TN * 16 * 2;
    auto load_b = [&](int i_) {
        const int st = i_ & 1;
        umma::mbar_arrive_expect_tx(&bfull[st], kTcDig * kBBytes);
#pragma unroll
        for (int pl = 0; pl < kTcDig; pl++)
            umma::bulk_g2s(Bs + st * Cfg::B_STAGE + pl * Cfg::B_PLANE,
                           Bu + ((int64_t)(st0 + i_) * kTcDig + pl) * s64 * 16, kBBytes, &bfull[st]);
        b_issued = i_;
    };

    if (warp < kTcProd) {
        // ---- producers: A digits.  Thread (row r, quarter kq) slices the
        // k-values 4 kq .. 4 kq + 3 of each 16-k step; a warp holds 16 rows x
        // 2 quarters, so that its stores of a plane fill two 128-byte core
        // matrices.  The gather runs three steps ahead in registers, every
        // load a whole step before its use: column data (step i + 3),
        // relative rows (i + 2), values (i + 1).
        const TcGather g{P.colbase + pos0, P.relbase + pos0, P.relidx, tile_cb, tile_rb, p0, c, gather_check(P)};
        const double *Zg = static_cast<const double *>(P.Z);
        const int r = (warp % 8) * 16 + (lane >> 1), kq = (warp / 8) * 2 + (lane & 1);
        const int E = rowE[r];
        double v[4];
        int64_t ab[4], cb[4], rb[4];
        int32_t ar[4];
        bool up[4];
        auto cols = [&](int i_) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (i_ < n) g.cols((st0 + i_) * 16 + kq * 4 + u, cb[u], rb[u]);
                else { cb[u] = -1; rb[u] = 0; }
            }
        };
        auto parts = [&](int i_) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (i_ < n) g.parts(r, (st0 + i_) * 16 + kq * 4 + u, cb[u], rb[u], ab[u], ar[u], up[u]);
                else { ab[u] = -1; ar[u] = 0; }
            }
            // bounds check (debug): an address outside the panels is dropped
            if (g.chk.on)
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (ab[u] >= 0 && !g.chk.ok(ab[u] + ar[u])) ab[u] = -1;
        };
        auto load = [&]() {
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = ab[u] >= 0 ? Zg[ab[u] + ar[u]] : 0.0;
        };
        if (n > 0) {
            cols(0);
            parts(0);
            load();
            cols(1);
            parts(1);
            cols(2);
        }
        for (int i_ = 0; i_ < n; i_++) {
            const int stage = i_ & 1, use = i_ >> 1;
            uint16_t *Ab = As + stage * Cfg::A_STAGE;
            if (i_ >= 2 && !umma::mbar_wait(&empty[stage], (uint32_t)((use - 1) & 1), mlim)) {
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
                uint16_t *dst = Ab + (r / 8) * 128 + (kq / 2) * 64 + (r % 8) * 8 + (kq % 2) * 4;
                store_plane4<0>(dst + 0 * Cfg::A_PLANE, lo, hi);
                store_plane4<1>(dst + 1 * Cfg::A_PLANE, lo, hi);
                store_plane4<2>(dst + 2 * Cfg::A_PLANE, lo, hi);
                store_plane4<3>(dst + 3 * Cfg::A_PLANE, lo, hi);
                store_plane4<4>(dst + 4 * Cfg::A_PLANE, lo, hi);
                store_plane4<5>(dst + 5 * Cfg::A_PLANE, lo, hi);
                store_plane4<6>(dst + 6 * Cfg::A_PLANE, lo, hi);
            }
            // release the step's operand first: the loads of later steps are
            // issued after the arrival, not between the stores and the fence
            umma::fence_proxy_async();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&full[stage]);
            load();            // values of step i + 1
            parts(i_ + 2);     // relative rows of step i + 2
            cols(i_ + 3);      // column data of step i + 3
            if (s_abort) break;
        }
    } else if (warp == kTcMmaWarp) {
        // ---- one thread issues the products once both operands of a step
        // are in place (and, at the start of a chunk, the epilogue has read
        // the previous one's group sums); it never waits for products
        if (lane == 0) {
            for (int i_ = 0; i_ < n; i_++) {
                const int stage = i_ & 1, use = i_ >> 1, ch = i_ / kTcFlush;
                const bool first = i_ % kTcFlush == 0;
                if (!umma::mbar_wait(&bfull[stage], (uint32_t)(use & 1), mlim) ||
                    !umma::mbar_wait(&full[stage], (uint32_t)(use & 1), mlim) ||
                    (first && ch > 0 && !umma::mbar_wait(&tmem_free, (uint32_t)((ch - 1) & 1), mlim))) {
                    s_abort = 1;
                    break;
                }
                umma::fence_after_sync();
                // plane i's descriptor = plane 0's + the plane offset in the start-address field
                const uint64_t ad0 = umma::smem_desc(umma::smem_u32(As + stage * Cfg::A_STAGE), 128, 256);
                const uint64_t bd0 = umma::smem_desc(umma::smem_u32(Bs + stage * Cfg::B_STAGE), 128, 256);
                digit_products<TN, Cfg::A_PLANE, Cfg::B_PLANE>(tmem, ad0, bd0, first);
                umma::commit(&empty[stage]);
                if (i_ % kTcFlush == kTcFlush - 1 || i_ == n - 1) umma::commit(&acc_full);
                if (s_abort) break;
            }
        }
        __syncwarp();
    } else if (warp == kTcCopyWarp) {
        // ---- one thread copies the Lhat digit planes of step i into the
        // stage of step i - 2 once the products of that step are done
        if (lane == 0) {
            for (int i_ = 0; i_ < n; i_++) {
                if (i_ >= 2 && !umma::mbar_wait(&empty[i_ & 1], (uint32_t)(((i_ >> 1) - 1) & 1), mlim)) {
                    s_abort = 1;
                    break;
                }
                load_b(i_);
                if (s_abort) break;
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: every chunk's exact fp32 group sums -> int64 (hi, lo)
        const int lb = 32 * (warp % 4), row = lb + lane, half = (warp / 4) & 1;
        for (int f = 0; f < nflush; f++) {
            if (!umma::mbar_wait(&acc_full, (uint32_t)(f & 1), mlim)) {
                s_abort = 1;
                break;
            }
            umma::fence_after_sync();
#pragma unroll 1
            for (int cb = half; cb < TN / 4; cb += 2) {
                uint32_t acc[kTcDig][4];
#pragma unroll
                for (int gq = 0; gq < kTcDig; gq++)
                    umma::tmem_ld4(tmem + ((uint32_t)lb << 16) + (uint32_t)(gq * TN + cb * 4), acc[gq]);
                umma::tmem_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 4; jj++) {
                    long long gv[kTcDig];
#pragma unroll
                    for (int gq = 0; gq < kTcDig; gq++) gv[gq] = (long long)__float2int_rn(__uint_as_float(acc[gq][jj]));
                    const long long h = (gv[0] << 16) + (gv[1] << 8) + gv[2];
                    const long long l = (gv[3] << 24) + (gv[4] << 16) + (gv[5] << 8) + gv[6];
                    long long *ph = Hi + (cb * 4 + jj) * kTcM + row, *pl = Lo + (cb * 4 + jj) * kTcM + row;
                    if (f == 0) {   // the first chunk writes, the later ones add
                        *ph = h;
                        *pl = l;
                    } else {
                        *ph += h;
                        *pl += l;
                    }
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
        if (warp == kTcMmaWarp && lane == 0) {
            umma::commit(&drain);
            umma::mbar_wait(&drain, 0u, mlim);
        }
        if (warp == kTcCopyWarp && lane == 0)   // the copies that may still be in flight
            for (int j = b_issued - 1 > 0 ? b_issued - 1 : 0; j <= b_issued; j++)
                umma::mbar_wait(&bfull[j & 1], (uint32_t)((j >> 1) & 1), mlim);
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (warp == kTcMmaWarp) umma::tmem_dealloc(tmem, Cfg::TCOLS);
        return;
    }
    umma::fence_after_sync();
    if (warp == kTcMmaWarp) umma::tmem_dealloc(tmem, Cfg::TCOLS);

    double *Zk = static_cast<double *>(P.Yout) + P.panel_off[K];
    // Y = -(A^{-1}_{C,C} Lhat): A digits on 2^(E - 1028 - 8i), Lhat digits on
    // 2^(F - 1029 - 8j), so the value is (hi 2^-16 + lo 2^-48) 2^(E + F - 2057)
    auto emit = [&](int row, int j, long long hi, long long lo) {
        const int sc = (rowE[row] - 1022) + (P.colexp[fc + j] - 1022) - 13;
        const double y = fixed_to_double(hi, lo, sc);
        Zk[(int64_t)j * ld + s + p0 + row] = -y;
        warp_uniform_atomic_max(&ymax[j], bexp(y));   // the lanes of a warp share column j
    };
    if (nsplit == 1) {
        for (int e = tid; e < kTcM * TN; e += kTcThreads) {
            const int row = e % kTcM, col = e / kTcM;
            if (p0 + row < c && n0 + col < s) emit(row, n0 + col, Hi[col * kTcM + row], Lo[col * kTcM + row]);
        }
    } else {
        // split k: the partial tile and the rows' exponents go to this CTA's
        // slab slot; k_tc_reduce sums the slots of the row tile afterwards
        long long *mine = slab + (int64_t)blockIdx.x * kTcSlot;
        for (int e = tid; e < kTcM * TN; e += kTcThreads) {
            mine[e] = Hi[e];
            mine[kTcM * 64 + e] = Lo[e];
        }
        int *re = reinterpret_cast<int *>(mine + 2 * kTcM * 64);
        for (int e = tid; e < kTcM; e += kTcThreads) re[e] = rowE[e];
        return;
    }
    __syncthreads();
    // column exponents of A^{-1}_{C,K} over all row tiles (used by the diagonal block)
    for (int j = tid; j < s; j += kTcThreads)
        if (ymax[j] > 0) atomicMax(&P.colexpY[fc + j], ymax[j]);
}

// Split-k reduction: one CTA per (row tile, 8 columns); each element sums
// the int64 words of the row tile's k-range slots in k order (exact) and
// forms A^{-1}_{C,K} = -(sum) on the row / column exponent grid.
// red[w] = {index of the group's first item, its slab slot, column block}.
template <int TN>
__global__ void __launch_bounds__(256) k_tc_reduce(const ProbDesc *__restrict__ descs,
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
    const int ncol = (s + TN - 1) / TN;
    const int nsplit = it.ntiles;
    const int p0 = (it.tile / nsplit / ncol) * kTcM;
    const long long *first = slab + (int64_t)rr.y * kTcSlot;
    const int *rowE = reinterpret_cast<const int *>(first + 2 * kTcM * 64);
    if (threadIdx.x < 8) ymax[threadIdx.x] = 0;
    __syncthreads();
    double *Zk = static_cast<double *>(P.Yout) + P.panel_off[K];
    const int row = threadIdx.x % kTcM;
    for (int jj = threadIdx.x / kTcM; jj < 8; jj += 256 / kTcM) {
        const int j = rr.z * 8 + jj;
        if (j >= s || p0 + row >= c) continue;
        const int ctj = j / TN, col = j % TN;
        long long hi = 0, lo = 0;
        for (int k2 = 0; k2 < nsplit; k2++) {
            const long long *sl = slab + ((int64_t)rr.y + ctj * nsplit + k2) * kTcSlot;
            hi += sl[col * kTcM + row];
            lo += sl[kTcM * 64 + col * kTcM + row];
        }
        const int sc = (rowE[row] - 1022) + (P.colexp[fc + j] - 1022) - 13;
        const double y = fixed_to_double(hi, lo, sc);
        Zk[(int64_t)j * ld + s + p0 + row] = -y;
        warp_uniform_atomic_max(&ymax[jj], bexp(y));   // the lanes of a warp share column j
    }
    __syncthreads();
    if (threadIdx.x < 8 && rr.z * 8 + (int)threadIdx.x < s && ymax[threadIdx.x] > 0)
        atomicMax(&P.colexpY[fc + rr.z * 8 + threadIdx.x], ymax[threadIdx.x]);
}

cudaError_t launch_tc_reduce(int tn, const ProbDesc *d, const Item *items, const int4 *red, int n,
                             const long long *slab, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (tn == 16) k_tc_reduce<16><<<n, 256, 0, st>>>(d, items, red, n, slab);
    else if (tn == 32) k_tc_reduce<32><<<n, 256, 0, st>>>(d, items, red, n, slab);
    else k_tc_reduce<64><<<n, 256, 0, st>>>(d, items, red, n, slab);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagonal block on tcgen05: the exact sums of (Lhat^T Y)(i, j) over one chunk
// of C rows for one column tile of K, added into K's per-entry int64 sums (the
// sums k_diag_fin turns into A^{-1}_KK = Dinv_K - Lhat^T Y).
//   A = Lhat^T: rows i of K (128 tensor-memory lanes, zero past s), k = rows q
//       of C -- the digit planes of Lhat are already stored in this operand
//       layout (they are the gather-GEMM's B), so one bulk copy per plane and
//       16-row step brings them in;
//   B = Y columns n0 .. n0 + TN - 1, k = q: 8 producer warps slice A^{-1}_{C,K}
//       (written by the gather-GEMM of this level) into digit planes on the
//       column exponents colexpY, integer operations only.
// Digit products grouped by i + j into exact fp32 sums in tensor memory,
// folded into int64 every 128 k, as in k_selinv_tc.  The A digits sit on the
// grid 2^(F - 1029 - 8i) of Lhat's columns, the B digits on 2^(E - 1028 - 8j).
// ---------------------------------------------------------------------------
constexpr int kDtProd = 8;                       // producer warps (digit planes of Y, 4 values per thread and step)
constexpr int kDtEpi = 8;                        // epilogue warps (tensor memory -> int64), two per lane quarter
constexpr int kDtMmaWarp = kDtProd + kDtEpi;     // one thread issues the products
constexpr int kDtCopyWarp = kDtMmaWarp + 1;       // one thread issues the Lhat digit copies
constexpr int kDtThreads = 32 * (kDtProd + kDtEpi + 2);

template <int TN> struct DtCfg {
    static constexpr int A_PLANE = kTcM * 16;
    static constexpr int B_PLANE = TN * 16;
    static constexpr int A_STAGE = kTcDig * A_PLANE;
    static constexpr int B_STAGE = kTcDig * B_PLANE;
    static constexpr uint32_t TCOLS = kTcDig * TN <= 128 ? 128u : (kTcDig * TN <= 256 ? 256u : 512u);
    static constexpr size_t SMEM =
        sizeof(uint16_t) * 2 * (size_t)(A_STAGE + B_STAGE) + sizeof(long long) * 2 * (size_t)kTcM * TN;
};
static_assert(4 * 64 <= 32 * kDtProd, "a producer thread per (column, 4-row quarter) of a 64-column tile");

// items: tile = (chunk * ncol + column tile) * nmt + m tile, ntiles = number
// of chunks; nmt = 1 for real supernodes.  CPLX: complex symmetric values,
// the real contraction over k' = 2q + part with the 2s rows of the complex
// Lhat operand (rows j: real part of row j of Lhat^T Y, rows s + j: its
// imaginary part; two m tiles when 2s > 128) and Y's (Re, Im) along k'; the
// sums go to (Re hi, Re lo, Im hi, Im lo) words per entry.
template <int TN, bool CPLX>
__global__ void __launch_bounds__(kDtThreads, 1) k_diag_tc(const ProbDesc *__restrict__ descs,
                                                           const Item *__restrict__ items, int nitems,
                                                           long long wait_limit) {
    grid_dep_wait();
    using Cfg = DtCfg<TN>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint16_t *As = reinterpret_cast<uint16_t *>(smem_raw);                // [2][7][A_PLANE]
    uint16_t *Bs = As + 2 * Cfg::A_STAGE;                                  // [2][7][B_PLANE]
    long long *Hi = reinterpret_cast<long long *>(Bs + 2 * Cfg::B_STAGE);  // [TN][128]
    long long *Lo = Hi + kTcM * TN;
    // full / afull: the producers' B and the bulk copies of A in a stage;
    // drain: every product issued before an abort is done
    __shared__ __align__(8) uint64_t full[2], afull[2], empty[2], acc_full, tmem_free, drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int colE[TN];

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
    const int kw = CPLX ? 2 * c : c;                    // k extent
    const int mrows = CPLX ? 2 * s : s;                 // rows of A (output rows)
    const int nsteps = (kw + 15) / 16;
    const int ncol = (s + TN - 1) / TN;
    const int nmt = (mrows + kTcM - 1) / kTcM;
    const int nch = it.ntiles;
    const int mt = it.tile % nmt;
    const int ct = (it.tile / nmt) % ncol, ch = it.tile / nmt / ncol;
    const int n0 = ct * TN, m0 = mt * kTcM;
    const int chunk = ((nsteps + nch - 1) / nch + kTcFlush - 1) / kTcFlush * kTcFlush;
    const int st0 = ch * chunk;
    const int st1 = st0 + chunk < nsteps ? st0 + chunk : nsteps;
    const int n = st1 > st0 ? st1 - st0 : 0;
    const int nflush = (n + kTcFlush - 1) / kTcFlush;
    const int64_t s64 = (mrows + 63) / 64 * 64;         // operand rows of a stored digit block
    const int arows = s64 - m0 < kTcM ? (int)(s64 - m0) : kTcM;

    if (tid == 0) s_abort = 0;
    // both A stages start at zero: the bulk copies fill rows < arows only
    for (int e = tid; e < 2 * Cfg::A_STAGE / 8; e += kDtThreads) reinterpret_cast<uint4 *>(As)[e] = make_uint4(0, 0, 0, 0);

    for (int j = tid; j < TN; j += kDtThreads) colE[j] = n0 + j < s ? P.colexpY[fc + n0 + j] : 0;
    if (tid == 0) {
        for (int st = 0; st < 2; st++) {
            umma::mbar_init(&full[st], kDtProd);
            umma::mbar_init(&afull[st], 1);     // the arrival that expects A's bytes
            umma::mbar_init(&empty[st], 1);
        }
        umma::mbar_init(&acc_full, 1);
        umma::mbar_init(&tmem_free, kDtEpi);
        umma::mbar_init(&drain, 1);
        umma::mbar_init_fence();
    }
    if (warp == kDtMmaWarp) {
        umma::tmem_alloc(&s_tmem, Cfg::TCOLS);
        umma::tmem_relinquish();
    }
    umma::fence_proxy_async();   // the zeroed A stages are seen by the tensor cores
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = s_tmem;
    int a_issued = -1;   // last step whose A copies the copy thread issued

    if (warp < kDtProd) {
        // ---- producers: thread (column r, quarter kq) slices rows 4 kq .. 4 kq + 3
        // of each 16-row step; a warp holds 16 columns x 2 quarters, so that its
        // stores of a plane fill two 128-byte core matrices.  The values of the
        // next step are loaded while this one is sliced.
        // Complex: the 4 k-values are (Re, Im) of rows q = 8 step + 2 kq and + 1.
        const int r = (warp % 4) * 16 + (lane >> 1), kq = (warp / 4) * 2 + (lane & 1);
        const bool act = r < TN;
        const int64_t ycol = P.panel_off[K] + (int64_t)(n0 + r) * ld + s;
        const bool colok = act && n0 + r < s;
        const int E = colok ? colE[r] : 0;
        double v[4];
        // Hermitian: Lhat^H Y = conj(Lhat^T conj(Y)), so the digits are those
        // of conj(Y) and the finisher conjugates the sums
        const bool cj = CPLX && P.herm;
        auto fetch = [&](int step) {
            if (CPLX) {
                const double2 *Yz = static_cast<const double2 *>(P.Z) + ycol;
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const int q = step * 8 + kq * 2 + u;
                    const double2 y = (colok && step < st1 && q < c) ? Yz[q] : make_double2(0.0, 0.0);
                    v[2 * u] = y.x;
                    v[2 * u + 1] = cj ? -y.y : y.y;
                }
            } else {
                const double *Yc = static_cast<const double *>(P.Z) + ycol;
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int q = step * 16 + kq * 4 + u;
                    v[u] = (colok && step < st1 && q < c) ? Yc[q] : 0.0;
                }
            }
        };
        if (n > 0) fetch(st0);
        for (int i_ = 0; i_ < n; i_++) {
            const int stage = i_ & 1, use = i_ >> 1;
            uint16_t *Bb = Bs + stage * Cfg::B_STAGE;
            if (i_ >= 2 && !umma::mbar_wait(&empty[stage], (uint32_t)((use - 1) & 1), mlim)) {
                s_abort = 1;
                break;
            }
            if (act) {
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
            umma::fence_proxy_async();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&full[stage]);
            if (i_ + 1 < n) fetch(st0 + i_ + 1);   // after the arrival (see k_selinv_tc)
            if (s_abort) break;
        }
    } else if (warp == kDtMmaWarp) {
        // ---- one thread issues the products once both operands are in place
        if (lane == 0) {
            for (int i_ = 0; i_ < n; i_++) {
                const int stage = i_ & 1, use = i_ >> 1, chk = i_ / kTcFlush;
                const bool first = i_ % kTcFlush == 0;
                if (!umma::mbar_wait(&afull[stage], (uint32_t)(use & 1), mlim) ||
                    !umma::mbar_wait(&full[stage], (uint32_t)(use & 1), mlim) ||
                    (first && chk > 0 && !umma::mbar_wait(&tmem_free, (uint32_t)((chk - 1) & 1), mlim))) {
                    s_abort = 1;
                    break;
                }
                umma::fence_after_sync();
                const uint64_t ad0 = umma::smem_desc(umma::smem_u32(As + stage * Cfg::A_STAGE), 128, 256);
                const uint64_t bd0 = umma::smem_desc(umma::smem_u32(Bs + stage * Cfg::B_STAGE), 128, 256);
                digit_products<TN, Cfg::A_PLANE, Cfg::B_PLANE>(tmem, ad0, bd0, first);
                umma::commit(&empty[stage]);
                if (i_ % kTcFlush == kTcFlush - 1 || i_ == n - 1) umma::commit(&acc_full);
                if (s_abort) break;
            }
        }
        __syncwarp();
    } else if (warp == kDtCopyWarp) {
        // ---- one thread copies the Lhat digit planes of step i into the
        // stage of step i - 2 once the products of that step are done
        if (lane == 0) {
            const uint16_t *Au = P.lhsu + P.lhsu_off[K] + (int64_t)(m0 / 8) * 128;
            const uint32_t aBytes = (uint32_t)(arows * 16 * 2);
            for (int i_ = 0; i_ < n; i_++) {
                if (i_ >= 2 && !umma::mbar_wait(&empty[i_ & 1], (uint32_t)(((i_ >> 1) - 1) & 1), mlim)) {
                    s_abort = 1;
                    break;
                }
                const int st = i_ & 1;
                umma::mbar_arrive_expect_tx(&afull[st], kTcDig * aBytes);
#pragma unroll
                for (int pl = 0; pl < kTcDig; pl++)
                    umma::bulk_g2s(As + st * Cfg::A_STAGE + pl * Cfg::A_PLANE,
                                   Au + ((int64_t)(st0 + i_) * kTcDig + pl) * s64 * 16, aBytes, &afull[st]);
                a_issued = i_;
                if (s_abort) break;
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue: every chunk's exact fp32 group sums -> int64 (hi, lo)
        const int lb = 32 * (warp % 4), row = lb + lane, half = (warp / 4) & 1;
        for (int f = 0; f < nflush; f++) {
            if (!umma::mbar_wait(&acc_full, (uint32_t)(f & 1), mlim)) {
                s_abort = 1;
                break;
            }
            umma::fence_after_sync();
#pragma unroll 1
            for (int cb = half; cb < TN / 8; cb += 2) {
                uint32_t acc[kTcDig][8];
#pragma unroll
                for (int gq = 0; gq < kTcDig; gq++)
                    umma::tmem_ld8(tmem + ((uint32_t)lb << 16) + (uint32_t)(gq * TN + cb * 8), acc[gq]);
                umma::tmem_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {
                    long long gv[kTcDig];
#pragma unroll
                    for (int gq = 0; gq < kTcDig; gq++) gv[gq] = (long long)__float2int_rn(__uint_as_float(acc[gq][jj]));
                    const long long h = (gv[0] << 16) + (gv[1] << 8) + gv[2];
                    const long long l = (gv[3] << 24) + (gv[4] << 16) + (gv[5] << 8) + gv[6];
                    long long *ph = Hi + (cb * 8 + jj) * kTcM + row, *pl = Lo + (cb * 8 + jj) * kTcM + row;
                    if (f == 0) {   // the first chunk writes, the later ones add
                        *ph = h;
                        *pl = l;
                    } else {
                        *ph += h;
                        *pl += l;
                    }
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
        // as in k_selinv_tc: drain this CTA's products and last bulk copies (bounded)
        if (tid == 0) atomicCAS(P.status, 0, SELINV_ERR_TIMEOUT);
        if (warp == kDtMmaWarp && lane == 0) {
            umma::commit(&drain);
            umma::mbar_wait(&drain, 0u, mlim);
        }
        if (warp == kDtCopyWarp && lane == 0)   // the copies that may still be in flight
            for (int j = a_issued - 1 > 0 ? a_issued - 1 : 0; j <= a_issued; j++)
                umma::mbar_wait(&afull[j & 1], (uint32_t)((j >> 1) & 1), mlim);
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (warp == kDtMmaWarp) umma::tmem_dealloc(tmem, Cfg::TCOLS);
        return;
    }
    umma::fence_after_sync();
    if (warp == kDtMmaWarp) umma::tmem_dealloc(tmem, Cfg::TCOLS);
    if (n == 0) return;
    // the chunk's exact sums into K's (cleared at the start of every call):
    // integer additions, so the order of chunks and column tiles does not matter
    long long *acc64 = P.dacc + (CPLX ? 4 : 2) * P.linv_off[K];
    for (int e = tid; e < kTcM * TN; e += kDtThreads) {
        const int ir = e % kTcM, col = e / kTcM, j = n0 + col, i = m0 + ir;
        if (i >= mrows || j >= s) continue;
        const long long hi = Hi[col * kTcM + ir], lo = Lo[col * kTcM + ir];
        unsigned long long *dst =
            CPLX ? reinterpret_cast<unsigned long long *>(acc64 + 4 * ((int64_t)j * s + (i < s ? i : i - s)) + (i < s ? 0 : 2))
                 : reinterpret_cast<unsigned long long *>(acc64 + 2 * ((int64_t)j * s + i));
        if (hi) atomicAdd(dst, (unsigned long long)hi);
        if (lo) atomicAdd(dst + 1, (unsigned long long)lo);
    }
}

cudaError_t launch_diag_tc(int tn, int cplx, const ProbDesc *d, const Item *items, int n, long long wait_limit,
                           cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (cplx) {
        if (tn == 32) k_diag_tc<32, true><<<n, kDtThreads, DtCfg<32>::SMEM, st>>>(d, items, n, wait_limit);
        else k_diag_tc<64, true><<<n, kDtThreads, DtCfg<64>::SMEM, st>>>(d, items, n, wait_limit);
    } else {
        if (tn == 32) k_diag_tc<32, false><<<n, kDtThreads, DtCfg<32>::SMEM, st>>>(d, items, n, wait_limit);
        else k_diag_tc<64, false><<<n, kDtThreads, DtCfg<64>::SMEM, st>>>(d, items, n, wait_limit);
    }
    return cudaGetLastError();
}

cudaError_t configure_tc_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_selinv_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<16>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_selinv_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<32>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_selinv_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<64>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_diag_tc<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DtCfg<32>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_diag_tc<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DtCfg<64>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_diag_tc<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DtCfg<32>::SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_diag_tc<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DtCfg<64>::SMEM);
    return e;
}

cudaError_t launch_selinv_tc(int tn, const ProbDesc *d, const Item *items, int n, long long *slab,
                             long long wait_limit, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (tn == 16) k_selinv_tc<16><<<n, kTcThreads, TcCfg<16>::SMEM, st>>>(d, items, n, slab, wait_limit);
    else if (tn == 32) k_selinv_tc<32><<<n, kTcThreads, TcCfg<32>::SMEM, st>>>(d, items, n, slab, wait_limit);
    else k_selinv_tc<64><<<n, kTcThreads, TcCfg<64>::SMEM, st>>>(d, items, n, slab, wait_limit);
    return cudaGetLastError();
}

}  // namespace selinv
