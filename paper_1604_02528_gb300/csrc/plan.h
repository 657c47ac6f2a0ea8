// Internal host-side structures of a plan (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <array>
#include <memory>
#include <utility>
#include <vector>

#include "common.cuh"

namespace selinv {

// Host allocator that leaves new elements default-initialized (no zeroing):
// for large index arrays that are filled completely right after allocation,
// so that their pages are first touched by the threads that fill them.
template <typename T> struct UninitAlloc : std::allocator<T> {
    template <typename U> struct rebind { using other = UninitAlloc<U>; };
    UninitAlloc() = default;
    template <typename U> UninitAlloc(const UninitAlloc<U> &) noexcept {}
    template <typename U> void construct(U *ptr) noexcept { ::new (static_cast<void *>(ptr)) U; }
    template <typename U, typename... A> void construct(U *ptr, A &&...a) {
        ::new (static_cast<void *>(ptr)) U(std::forward<A>(a)...);
    }
};
template <typename T> using fill_vector = std::vector<T, UninitAlloc<T>>;

struct PlanData {
    int32_t n = 0, ns = 0;
    int device = -1;   // CUDA device of the plan's device arrays (set by ensure_device)
    selinv_opts opts{};
    bool tuned[3] = {false, false, false};   // autotuning done, per selinv_dtype
    // host arrays (kept for inspection and schedule building)
    std::vector<int32_t> super_ptr, sparent, rows, level, level_list;
    std::vector<int32_t> seg_owner, seg_start, seg_coloff, ntiles;
    fill_vector<int32_t> relidx;
    std::vector<int64_t> rowptr, panel_off, seg_ptr, rel_ptr, level_ptr, linv_off, part_off;
    std::vector<int64_t> part_off_all;  // split-partial offsets disjoint over all levels (persistent schedule)
    fill_vector<int64_t> colbase, relbase;  // per row-list position
    std::vector<int64_t> lhs_off;           // digit-plane offsets (tensor-core path)
    std::vector<int64_t> lhsu_off;          // the same in the tcgen05 operand layout
    std::vector<int64_t> lhsuz_off;         // complex Lhat operand (2s rows, 2c k) in that layout
    std::vector<int64_t> tile_base;         // prefix sums of the 64-row tiles of each supernode
    std::vector<int64_t> linvd_off;         // digit planes of L_KK^{-1} (tensor-core path)
    // subset selection: the supernodes that run (empty: all) and the panel
    // positions of the selected entries
    std::vector<uint8_t> active;
    std::vector<int64_t> sel_pos;
    int64_t sel_version = 0;
    int64_t *d_sel_pos = nullptr;
    int nlevels = 0;
    int64_t nnz = 0, linv_total = 0, part_max = 1, part_all = 1, lhs_total = 0, lhsu_total = 0, tile_total = 0, linvd_total = 0,
            lhsuz_total = 0;
    // device copies
    int32_t *d_super_ptr = nullptr, *d_sparent = nullptr, *d_rows = nullptr, *d_relidx = nullptr;
    int64_t *d_rowptr = nullptr, *d_panel_off = nullptr, *d_colbase = nullptr, *d_relbase = nullptr;
    int64_t *d_linv_off = nullptr, *d_part_off = nullptr, *d_part_off_all = nullptr, *d_lhs_off = nullptr, *d_lhsu_off = nullptr, *d_tile_base = nullptr,
            *d_lhsuz_off = nullptr;
    int64_t *d_linvd_off = nullptr;
    int64_t *d_seg_ptr = nullptr;      // owner segments (push schedule)
    int32_t *d_seg_start = nullptr;
    int *d_status = nullptr;
    void release_device();
};

// Numeric scratch of one problem: Dinv/Lhat panels, L_KK^{-1} blocks, split
// partials of the diagonal blocks, per-supernode tile counters and
// completion flags, and one more panel-sized buffer (adjoint working copy).
// Makes `dev` the current device for a scope and restores the caller's
// device afterwards (dev < 0: nothing to do).
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev) {
        if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev)
            switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

struct Workspace {
    int device = -1;           // device the buffers below live on
    void *LD = nullptr, *Linv = nullptr, *partial = nullptr, *work = nullptr;
    void *partial_all = nullptr;  // persistent schedule: supernodes of every level in flight at once
    int *counter = nullptr, *done = nullptr;
    uint16_t *lhs = nullptr;   // fp16 digit planes of Lhat
    uint16_t *lhsu = nullptr;  // the same in the tcgen05 operand layout (zero padding)
    int *colexp = nullptr;     // [n]
    int *colexpY = nullptr;    // [n], zero between calls
    long long *dacc = nullptr; // [2 * linv_total] (complex: 4 *), zero between calls
    int *colexpZ = nullptr;    // [n], rewritten for every column in every call
    int *ticket = nullptr;     // work-item ticket of the persistent schedule
    uint16_t *linvd = nullptr; // digit planes of L_KK^{-1}
    int *linvexp = nullptr;    // [n]
    long long *yacc = nullptr; // [2 * nnz] (real problems with tensor-core supernodes), zero between calls
    int *tcount = nullptr;     // [tile_total], zero between calls
    void *LDu = nullptr;       // LU form: Uhat^T panels
    void *Vt = nullptr;        // LU form: (U_KK^T)^{-1} blocks
    size_t bytes_elem = 0;
    std::vector<std::pair<void *, size_t>> owned;   // every buffer above, with its size
    int ensure(const PlanData &p, int dtype);
    int ensure_lu(const PlanData &p);
    int ensure_persistent(const PlanData &p);
    void release();
};

// Device buffers through the cache of released workspaces (devmem.cu):
// dev_alloc hands out a cached buffer of exactly `bytes` or allocates one;
// dev_release caches the buffer (the caller has synchronized the device).
cudaError_t dev_alloc(void **ptr, size_t bytes);
void dev_release(void *ptr, size_t bytes);

// launch kinds
enum { KL_LINV = 0, KL_LHAT = 1, KL_SELINV = 2, KL_DIGITS = 3, KL_SELINV_OZ = 4, KL_DIAG = 5, KL_LINV_DIGITS = 6,
       KL_LHAT_OZ = 7, KL_PERSIST = 8, KL_SELINV_TC = 9, KL_TC_REDUCE = 10, KL_DIAG_FIN = 11,
       KL_PUSH_DIAG = 12, KL_PUSH = 13, KL_DINV = 14, KL_DIAG_TC = 15, KL_SELINV_TINY = 16, KL_NKINDS = 17 };

// tensor-core (FP64-exact) contraction applies to real problems with s >= kOzMinS;
// fast_contraction 1 runs the gather-GEMM on tcgen05, 2 on mma.sync
constexpr int kOzMinS = 1;
inline bool oz_eligible(int dtype, int s, const selinv_opts &o) {
    return o.fast_contraction && dtype == SELINV_F64 && s >= std::max(kOzMinS, o.oz_min_s);
}
constexpr int kTcRows = 128;   // rows of C per tcgen05 item
constexpr int kTcChunkSteps = 8;   // k16 steps per exact fp32 chunk of the tensor-core kernels (k-ranges are whole chunks)
constexpr int kTcWide = 128;   // launch bucket of the transposed tcgen05 kernel (supernodes wider than 64)
constexpr int kTcWideRows = 64;   // rows of C per item of that kernel
constexpr int kAsmChunk = 1024;   // entries of an update matrix per extend-add item
constexpr int kTopSupernodes = 16;   // level schedule: the top levels (up to this many supernodes) normalized first
constexpr int kMidSupernodes = 256;  // ... and the levels up to this many normalized in the side stream's first phase

struct Launch {
    int kind;    // KL_*
    int dtype;
    int bucket;
    int64_t off;
    int count;
    int level;
    int side = 0;   // 1, 2: issued on the schedule's side stream (normalization phases of the lower levels)
};

struct Schedule {
    bool valid = false;
    int mode = -1;
    const void *key_L = nullptr, *key_D = nullptr, *key_Z = nullptr, *key_Z2 = nullptr;
    int key_dtype = -1;
    std::vector<ProbDesc> h_descs;
    std::vector<Item> h_items;
    std::vector<int2> h_work;
    std::vector<int8_t> h_buckets;  // per item of the persistent launches
    std::vector<int4> h_red;        // split-k reductions: (group's first item, its slab slot, 8-column block)
    std::vector<Launch> launches;
    std::vector<void *> reset_ptr;  // memsets issued before the persistent launches
    std::vector<size_t> reset_bytes;
    std::vector<void *> pre_ptr;    // memsets issued at the start of every call
    std::vector<size_t> pre_bytes;
    ProbDesc *d_descs = nullptr;
    Item *d_items = nullptr;
    int2 *d_work = nullptr;
    int8_t *d_buckets = nullptr;
    int4 *d_red = nullptr;
    int *ticket = nullptr;
    long long *tcslab = nullptr;  // split-k partial tiles of the tcgen05 launches, one per CTA
    long long spin_limit = 0;   // bound of every device wait of the schedule's kernels
    int wait_on_unset = 0;
    cudaGraphExec_t graph = nullptr;
    // selinv_numeric_host's captured call and the buffers it was captured for
    cudaGraphExec_t graph_host = nullptr;
    std::array<const void *, 6> host_key{};
    // level schedule: the side stream that normalizes the lower levels'
    // supernodes while the main stream traverses the top levels, and the
    // launch before which the main stream waits for it (-1: none)
    int join_at = -1, join_at2 = -1;   // the second join: three phases
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_mid = nullptr;
    void release();
};

// copy streams and events of selinv_numeric_host
struct HostPipe {
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t ev_top = nullptr, ev_mid = nullptr, ev_rest = nullptr, ev_done = nullptr, ev_in_done = nullptr;
    std::vector<cudaEvent_t> ev_grp;
    void release();
};

struct BatchEntry {
    int mode = -1;
    std::vector<struct selinv_plan_s *> plans;
    std::vector<int> dtypes;
    std::vector<const void *> L, D;
    std::vector<void *> Z;
    std::vector<int64_t> sel_version;   // each plan's selection when the schedule was built
    Schedule sched;
};

size_t elem_size(int dtype);
int ensure_device(PlanData &p);
ProbDesc make_desc(const PlanData &p, Workspace &w, int dtype, const void *L, const void *D, void *Z,
                   bool persistent);
// split_norm: in the level schedule, normalize the lower levels on the side
// stream (see plan.cu); false keeps every launch on one stream
int build_schedule(Schedule &S, const std::vector<const PlanData *> &plans,
                   const std::vector<ProbDesc> &descs, int mode, bool split_norm = true);
int run_schedule(Schedule &S, cudaStream_t st, bool use_graph);
// kernel-to-kernel edges of a captured graph -> programmatic (see plan.cu)
cudaError_t programmatic_edges(cudaGraph_t g);
cudaError_t launch_with(const Schedule &S, const Launch &L, const ProbDesc *d, cudaStream_t st);

// factorization / adjoint state
struct FactorDesc {
    const int32_t *super_ptr;
    const int32_t *sparent;
    const int64_t *rowptr;
    const int32_t *rows;
    const int64_t *panel_off;
    const int64_t *u_off;     // [ns+1] update matrix of K: c x c column-major at U + u_off[K]
    const int32_t *chpos;     // per row-list entry of C_K: its position in rows(parent(K))
    void *U;                  // update matrices (element type of the factorization)
    void *L;
    void *D;
    int *status;
    int herm;                 // complex Hermitian: A = L D L^H
};

struct FactorData {
    int32_t n = -1;
    int64_t nnzA = 0;
    std::vector<int64_t> a_pos;       // panel position of every stored entry of A
    int64_t *d_a_pos = nullptr;
    // launch lists, leaves first
    std::vector<int2> h_tiles;        // (J, row tile) per level
    std::vector<int> h_js;            // J per level
    std::vector<int64_t> tile_lptr, j_lptr;
    int2 *d_tiles = nullptr;
    int *d_js = nullptr;
    // update matrices (multifrontal hand-off from child to parent; shared
    // with the selected-inversion adjoint)
    std::vector<int64_t> u_off;
    std::vector<int32_t> chpos;
    std::vector<int2> asm_items;      // (child, kAsmChunk-entry chunk) per level and child rank
    std::vector<int64_t> asm_lptr;    // [level * npass + rank]
    int npass = 1;
    std::vector<int4> uitems;         // (K, row tile, column tile) of the lower c x c, per level
    std::vector<int64_t> u_lptr;
    int2 *d_asm = nullptr;
    int4 *d_uitems = nullptr;
    int64_t *d_uoff = nullptr;
    int32_t *d_chpos = nullptr;
    void *U = nullptr;
    size_t U_bytes = 0;
    FactorDesc *d_desc = nullptr;
    const void *key_L = nullptr, *key_D = nullptr;
    int key_dtype = -1;
    // adjoint state
    void *adj = nullptr;
};


}  // namespace selinv

struct selinv_plan_s {
    selinv::PlanData data;
    std::vector<selinv::Workspace> ws;  // ws[0]: single calls; ws[1..]: batch items
    selinv::Schedule single;
    selinv::Schedule lu;                // the LU form (selinv_numeric_lu)
    selinv::HostPipe host;              // selinv_numeric_host's copy streams
    std::vector<selinv::BatchEntry> batch_cache;
    selinv::FactorData *factor = nullptr;
    cudaStream_t last_stream = nullptr;
    ~selinv_plan_s();
};

namespace selinv {
void factor_release(selinv_plan_s *plan);
void adjoint_release(void *adj);
int factor_tables(selinv_plan_s *plan);
}
