// kernels.h -- host-side launchers of the NI-ORCA stages (internal).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace niorca {

// Per-call work memory, carved from one pool allocation.
struct Work {
    int n = 0, m = 0;
    int ntiles = 0;          // relabel tiles of RL_TILE vertices
    int2 *vinfo = nullptr;   // old id -> (new id, degree)
    int *perm = nullptr;     // new id -> old id
    int *chist = nullptr;    // class histogram, NCLASS x ntiles (class-major)
    int *coff = nullptr;     // exclusive scan of chist
    int *nrow = nullptr;     // relabelled offsets, n + 1
    int *split = nullptr;    // scan input: degree of each new id
    int4 *rinfo = nullptr;   // {row start, split, row end, 0} per new id
    int *ncol = nullptr;     // relabelled neighbours, m
    int *tcnt = nullptr;     // triangle count of each out-entry (u, v), u < v; m ints in a region of 8 m bytes
    VAcc *vacc = nullptr;    // per-vertex accumulators, n
    int *scan_part = nullptr;// scan block partials
    int *lists = nullptr;    // heavy-vertex lists, 6 x n
    int *counters = nullptr; // list lengths and flags, 16 ints
    int *status = nullptr;   // device status word (not part of the carve)
    int num_sms = 0;
    int tune[11] = {16, 8, 8, 8, 8, 32, 1536, 64, 1152, 8192, 12288};  // see TuneIndex
    int induced = 0;         // write induced instead of non-induced counts
};

// Runtime tuning knobs (niorca_set_tuning): CTAs per SM of the persistent
// warp-tier kernels, and the thresholds that route vertices to a warp or a CTA.
enum TuneIndex {
    TUNE_GRID_RELABEL = 0,   // k_relabel_rows_warp CTAs per SM
    TUNE_GRID_TRI = 1,       // k_tri_warp
    TUNE_GRID_AGG = 2,       // k_agg_warp
    TUNE_GRID_C4 = 3,        // k_c4_warp
    TUNE_GRID_SOLVE = 4,     // k_solve
    TUNE_LONG_ROW_CLASS = 5, // degree class from which a row is relabelled by a whole CTA
    TUNE_C4_WARP_MAXW = 6,   // largest wedge count W of a 4-cycle root kept in one warp (<= 1536)
    TUNE_WARP_MAXD = 7,      // largest out-degree of a triangle root kept in one warp (<= 64)
    TUNE_TRI_BITS_MAXD = 8,  // largest out-degree of a CTA-tier triangle root that keeps the bit matrix R (<= 1152)
    TUNE_TRI_HASH_MAXD = 9,  // largest out-degree of a CTA-tier triangle root that hashes N+(u) (<= 8192)
    TUNE_C4_TEAM_MINW = 10,  // 4-cycle roots with more wedges than this go to the key-tiled tier (<= 12288)
    TUNE_COUNT = 11
};

// Indices into Work::counters.
// The triangle and aggregate heavy lists hold two tiers each: CTA-sized
// roots from the front (CNT_*_HEAVY), the largest from the back (CNT_*_BIG).
// The *_NEXT entries are the work counters of the CTA tiers: each CTA takes
// its next root from the queue's counter, so a CTA that starts late (or a
// root that takes long) leaves no other CTA idle.
enum { CNT_TRI_HEAVY = 0, CNT_AGG_HEAVY = 1, CNT_C4_CTA = 2, CNT_C4_TEAM = 3, CNT_DMAX = 4, CNT_C4_MID = 5,
       CNT_C4_MIDP = 6, CNT_TRI_BIG = 7, CNT_AGG_BIG = 8, CNT_C4_WBIG = 9, CNT_C4_TILED_NEXT = 10,
       CNT_TRI_CTA_NEXT = 11, CNT_TRI_BIG_NEXT = 12, CNT_AGG_CTA_NEXT = 13, CNT_AGG_BIG_NEXT = 14,
       CNT_C4_MID_NEXT = 15, CNT_C4_MIDP_NEXT = 16, CNT_C4_CTA_NEXT = 17, NCOUNTERS = 32 };

// The next item of a work queue, for the whole CTA: thread 0 takes it from
// the queue's counter, every thread returns the same index.
__device__ __forceinline__ int cta_next(int *ctr) {
    __shared__ int s_item;
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1);
    __syncthreads();
    return s_item;
}

// Programmatic dependent launch: every kernel of the library is launched
// with launch_pdl, so that the next kernel on the stream is set up while
// the CTAs of the one before it drain (which hides most of the launch gap
// between the short kernels of a small graph), and begins with pdl_begin:
// it waits until the kernel before it has completed and its writes are
// visible, before touching memory. No kernel triggers its dependents early:
// CTAs of the next kernel waiting on SMs from the start of a kernel made
// the ER n = 1e6 call 35% slower.
__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... P, class... A>
void launch_pdl(void (*kernel)(P...), unsigned grid, unsigned threads, size_t smem, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// CTAs of `kernel` (launched with `threads` threads and `smem` bytes of
// dynamic shared memory) that one SM holds at once: the size of a
// persistent grid is SMs times this.
int resident_ctas(const void *kernel, int threads, size_t smem);

// Whether the degree pass found a degree above MAX_DEGREE. NIORCA_EOVERFLOW
// is then recorded already, and every kernel after the relabelling returns
// at once: their fixed-size shared buffers and 32-bit partial sums rely on
// the bound (Sec. 3 bounds the work by the largest degree; the bound itself
// is this library's choice, see MAX_DEGREE).
__device__ __forceinline__ bool degree_overflow(const int *counters) {
    return *reinterpret_cast<const volatile int *>(counters + CNT_DMAX) > MAX_DEGREE;
}

constexpr int RL_TILE = 2048;        // vertices per class-histogram tile
constexpr int SCAN_TILE = 4096;      // elements per scan block
constexpr int LONG_ROW_CLASS = 32;   // deg_class(512): rows from here on get a CTA each

size_t scan_partials(long long len);
void launch_exclusive_scan(const int *in, int *out, long long len, bool write_total, int *part,
                           cudaStream_t st);

void launch_relabel(const int *rowptr, const int *colidx, Work &w, cudaStream_t st);
void launch_stage1(Work &w, cudaStream_t st);
void launch_stage2(Work &w, cudaStream_t st);
void launch_cycle4(Work &w, cudaStream_t st);
void launch_solve(Work &w, long long *out, cudaStream_t st);
void launch_validate(const int *rowptr, const int *colidx, int n, int m, int *status, int num_sms,
                     cudaStream_t st);

// Kernel ids for the optional per-kernel event timing and launch counting.
enum KernelId {
    K_CLASS_HIST, K_SCAN, K_CLASS_SCATTER, K_RELABEL_WARP, K_RELABEL_CTA, K_BATCH_SETUP,
    K_TRI_WARP, K_TRI_CTA, K_AGG_WARP, K_AGG_CTA, K_C4_WARP, K_C4_CTA, K_C4_PLAN, K_C4_TILED,
    K_SOLVE, K_VALIDATE, K_C4_MID, K_TRI_BIG, K_AGG_BIG, K_C4_WARP_BIG, K_C4_WEDGE_LEN, K_COUNT
};
const char *kernel_name(int id);

// Called after every kernel launch: counts it and, when timing is on,
// records an event on the launching stream.
void after_launch(cudaStream_t st, int id);

}  // namespace niorca
