// cycle4.cu -- 4-cycles through every vertex (psi_8).
//
// The paper obtains psi_8 from Stage III's `common[z]` array: for a fixed x,
// common[z] counts the 2-paths x-y-z, and f_8^12 sums common[z] - 1 over the
// paths (Table 1, Fig. 3d; Appendix, o8). Per vertex this equals
// psi_8(x) = sum over w != x of C(c_xw, 2), c_xw = |N(x) ∩ N(w)|.
// Here every 4-cycle is built once, from its highest vertex u (in the
// degree order of the relabelling): wedges u - v - w with v < u and w < u
// are counted per end point w in a hash table, c_w = number of such wedges;
// then
//   u gets sum_w C(c_w, 2), w gets C(c_w, 2),
//   each middle vertex v gets sum over its wedges of (c_w - 1).
// The wedges through v are the entries of row v below u; the whole row is
// streamed (it is read anyway) and filtered, so there is no dependent search.
// Roots are routed by the bound UB = sum over v of (d_v - 1) >= wedges:
// one warp with a 1024-slot shared table, four warps with 4096 slots, a
// 512-thread CTA with 16384 slots, or a CTA with a dense count row in global
// memory. Each table is emptied once per CTA; afterwards a root empties only
// the slots it filled (kept in a `touched` list).
#include "kernels.h"

namespace niorca {

constexpr int CW_WARPS = 4;
constexpr int CW_SLOTS = 1024;
constexpr int CW_MAXUB = 768;
constexpr int CM_THREADS = 128;
constexpr int CM_SLOTS = 4096;
constexpr int CM_MAXUB = 3072;
constexpr int CC_THREADS = 512;
constexpr int CC_SLOTS = 16384;
constexpr int CC_MAXUB = 12288;
constexpr int CG_THREADS = 1024;

__device__ __forceinline__ long long c2(long long c) { return c * (c - 1) / 2; }

// Segment table of in-neighbour chunk cb of root u in the calling warp: the
// rows of v = ncol[b + cb + lane] concatenated; returns the total length.
__device__ __forceinline__ int wedge_chunk(const Graph &g, int b, int din, int cb, int *sst, int *spre, int *vout) {
    const int lane = lane_id();
    const int p = cb + lane;
    int v = -1, st = 0, len = 0;
    if (p < din) {
        v = g.ncol[b + p];
        const int4 rv = g.rinfo[v];
        st = rv.x;
        len = rv.z - rv.x;
    }
    const int incl = warp_inclusive_scan(len);
    sst[lane] = st;
    spre[lane] = incl - len;
    *vout = v;
    const int total = __shfl_sync(FULL, incl, 31);
    __syncwarp();
    return total;
}

// Walks the wedges of root u (in-neighbours b .. b + din of row u), one warp
// per chunk of 32 in-neighbours (chunks c0, c0 + cstep, ...): f(q, w) for each
// entry w < u of their rows (q: lane that owns v), then done(v) per chunk.
template <class F, class D>
__device__ __forceinline__ void walk_wedges(const Graph &g, int u, int b, int din, int c0, int cstep, int *sst,
                                            int *spre, F f, D done) {
    const int lane = lane_id();
    for (int cb = c0 * 32; cb < din; cb += cstep * 32) {
        int v;
        const int total = wedge_chunk(g, b, din, cb, sst, spre, &v);
        seg_expand<4>(g.ncol, sst, spre, total, lane, 32, [&](int q, int, int w) {
            if (w < u) f(q, w);
        });
        __syncwarp();
        done(v);
        __syncwarp();
    }
}

// The same walk shared by all warps of a CTA: every warp builds the segment
// table of each chunk and takes the elements wid * 32 + lane, stride nw * 32.
// With DONE, warp 0 calls done(v) after the whole CTA finished the chunk.
template <bool DONE, class F, class D>
__device__ __forceinline__ void walk_wedges_cta(const Graph &g, int u, int b, int din, int wid, int nw, int *sst,
                                                int *spre, F f, D done) {
    const int lane = lane_id();
    for (int cb = 0; cb < din; cb += 32) {
        int v;
        const int total = wedge_chunk(g, b, din, cb, sst, spre, &v);
        seg_expand<4>(g.ncol, sst, spre, total, wid * 32 + lane, nw * 32, [&](int q, int, int w) {
            if (w < u) f(q, w);
        });
        if (DONE) {
            __syncthreads();
            if (wid == 0) done(v);
            __syncthreads();
        } else {
            __syncwarp();
        }
    }
}

// Counts `key`; returns the slot when this call inserted it, else -1.
__device__ __forceinline__ int hcount_add_new(int *keys, int *cnts, unsigned mask, int key) {
    unsigned s = hash_slot(key, mask);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        int k = keys[s];
        if (k == -1) {
            const int prev = atomicCAS(&keys[s], -1, key);
            if (prev == -1) { atomicAdd(&cnts[s], 1); return (int)s; }
            k = prev;
        }
        if (k == key) { atomicAdd(&cnts[s], 1); return -1; }
        s = (s + 1) & mask;
    }
    return -1;
}

// Shared-memory view of one root's table (keys, counts, filled slots).
struct C4Tab {
    int *hk, *hc, *touched, *ntouched;
    unsigned mask;
};

// Counts all wedges of u into the table and credits every 4-cycle rooted at
// u. Every thread of the group (one warp, or a CTA with CTA = true) calls it.
// pv holds the per-middle-vertex sums of one chunk (per warp, or shared by
// the CTA).
template <bool CTA>
__device__ __forceinline__ void c4_root(const Graph &g, VAcc *vacc, int u, int b, int din, const C4Tab &T, int wid,
                                        int nw, int tid, int nthreads, int *sst, int *spre, long long *pv,
                                        int *any_cycle) {
    const int lane = lane_id();
    auto sync = [] {
        if (CTA) __syncthreads(); else __syncwarp();
    };
    auto insert = [&](int, int w) {
        const int slot = hcount_add_new(T.hk, T.hc, T.mask, w);
        if (slot >= 0) T.touched[atomicAdd(T.ntouched, 1)] = slot;
    };
    if (CTA) walk_wedges_cta<false>(g, u, b, din, wid, nw, sst, spre, insert, [](int) {});
    else walk_wedges(g, u, b, din, 0, 1, sst, spre, insert, [](int) {});
    sync();
    const int nt = *T.ntouched;
    long long su = 0;
    for (int i = tid; i < nt; i += nthreads) {
        const int slot = T.touched[i];
        const int c = T.hc[slot];
        if (c >= 2) {
            su += c2(c);
            add64(&vacc[T.hk[slot]].C4, c2(c));
        }
    }
    su = warp_sum(su);
    if (lane == 0 && su) {
        add64(&vacc[u].C4, su);
        *any_cycle = 1;
    }
    sync();
    if (*any_cycle) {   // middle vertices, only when some cycle is rooted at u
        if (tid < 32) pv[tid] = 0;
        sync();
        auto middle = [&](int q, int w) {
            const int c = hcount_get(T.hk, T.hc, T.mask, w);
            if (c > 1) atomicAdd((unsigned long long *)&pv[q], (unsigned long long)(c - 1));
        };
        auto flush = [&](int v) {
            const long long x = pv[lane];
            if (x) add64(&vacc[v].C4, x);
            pv[lane] = 0;
        };
        if (CTA) walk_wedges_cta<true>(g, u, b, din, wid, nw, sst, spre, middle, flush);
        else walk_wedges(g, u, b, din, 0, 1, sst, spre, middle, flush);
    }
    sync();
    for (int i = tid; i < nt; i += nthreads) {
        const int slot = T.touched[i];
        T.hk[slot] = -1;
        T.hc[slot] = 0;
    }
    sync();
    if (tid == 0) {
        *T.ntouched = 0;
        *any_cycle = 0;
    }
    sync();
}

struct C4WarpSmem {
    int hk[CW_SLOTS];
    int hc[CW_SLOTS];
    int touched[CW_MAXUB];
    int sst[32];
    int spre[32];
    long long pv[32];
    int ntouched;
    int any_cycle;
};

// One warp per root with UB <= maxub (<= CW_MAXUB); larger roots are queued.
__global__ void __launch_bounds__(CW_WARPS * 32) k_c4_warp(Graph g, VAcc *vacc, int *lists, int *counters,
                                                           int maxub) {
    __shared__ C4WarpSmem sm_all[CW_WARPS];
    C4WarpSmem &S = sm_all[threadIdx.x >> 5];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int *mid_list = lists + 2 * (size_t)g.n;
    int *cta_list = lists + 3 * (size_t)g.n;
    int *glob_list = lists + 4 * (size_t)g.n;
    for (int i = lane; i < CW_SLOTS; i += 32) { S.hk[i] = -1; S.hc[i] = 0; }
    if (lane == 0) { S.ntouched = 0; S.any_cycle = 0; }
    __syncwarp();
    const C4Tab T{S.hk, S.hc, S.touched, &S.ntouched, CW_SLOTS - 1};
    for (int u = gw; u < g.n; u += nw) {
        const int4 ru = g.rinfo[u];
        const int b = ru.x, din = ru.y - ru.x;
        if (din < 2) continue;
        long long ub = 0;
        for (int p = lane; p < din; p += 32) {
            const int4 rv = g.rinfo[g.ncol[b + p]];
            ub += rv.z - rv.x - 1;
        }
        ub = warp_sum(ub);
        if (ub < 2) continue;
        if (ub > maxub) {
            if (lane == 0) {
                if (ub > CC_MAXUB) glob_list[atomicAdd(&counters[CNT_C4_GLOBAL], 1)] = u;
                else if (ub > CM_MAXUB) cta_list[atomicAdd(&counters[CNT_C4_CTA], 1)] = u;
                else mid_list[atomicAdd(&counters[CNT_C4_MID], 1)] = u;
            }
            continue;
        }
        c4_root<false>(g, vacc, u, b, din, T, 0, 1, lane, 32, S.sst, S.spre, S.pv, &S.any_cycle);
    }
}

// Roots from a queue, one CTA each, table of SLOTS entries in dynamic
// shared memory (emptied once per CTA).
template <int THREADS, int SLOTS, int MAXUB>
__device__ __forceinline__ void c4_queue(const Graph &g, VAcc *vacc, const int *list, int count) {
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int NW = THREADS / 32;
    int *hk = reinterpret_cast<int *>(dsm);
    int *hc = hk + SLOTS;
    int *touched = hc + SLOTS;
    int *segs = touched + MAXUB;       // NW x 64 ints: sst, spre per warp
    long long *pv = reinterpret_cast<long long *>(segs + NW * 64);   // 32, shared by the CTA
    int *flags = reinterpret_cast<int *>(pv + 32);                  // ntouched, any_cycle
    const int wid = threadIdx.x >> 5;
    int *sst = segs + wid * 64;
    int *spre = sst + 32;
    for (int i = threadIdx.x; i < SLOTS; i += THREADS) { hk[i] = -1; hc[i] = 0; }
    if (threadIdx.x == 0) { flags[0] = 0; flags[1] = 0; }
    __syncthreads();
    const C4Tab T{hk, hc, touched, &flags[0], SLOTS - 1};
    for (int h = blockIdx.x; h < count; h += gridDim.x) {
        const int u = list[h];
        const int4 ru = g.rinfo[u];
        c4_root<true>(g, vacc, u, ru.x, ru.y - ru.x, T, wid, NW, threadIdx.x, THREADS, sst, spre, pv, &flags[1]);
    }
}

constexpr size_t cq_smem(int threads, int slots, int maxub) {
    return (size_t)(2 * slots + maxub + (threads / 32) * 64 + 64 + 4) * 4;
}
constexpr size_t CM_SMEM = cq_smem(CM_THREADS, CM_SLOTS, CM_MAXUB);
constexpr size_t CC_SMEM = cq_smem(CC_THREADS, CC_SLOTS, CC_MAXUB);

__global__ void __launch_bounds__(CM_THREADS) k_c4_mid(Graph g, VAcc *vacc, const int *lists, const int *counters) {
    c4_queue<CM_THREADS, CM_SLOTS, CM_MAXUB>(g, vacc, lists + 2 * (size_t)g.n, counters[CNT_C4_MID]);
}

__global__ void __launch_bounds__(CC_THREADS) k_c4_cta(Graph g, VAcc *vacc, const int *lists, const int *counters) {
    c4_queue<CC_THREADS, CC_SLOTS, CC_MAXUB>(g, vacc, lists + 3 * (size_t)g.n, counters[CNT_C4_CTA]);
}

// Zero the dense rows of the global tier (only when that tier has work).
__global__ void k_c4_zero_dense(int *dense, long long n, int slots, const int *counters) {
    const int nh = counters[CNT_C4_GLOBAL];
    if (nh == 0) return;
    const long long rows = nh < slots ? nh : slots;
    const long long total = rows * n;
    int4 *d4 = reinterpret_cast<int4 *>(dense);
    const long long n4 = total / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        d4[i] = make_int4(0, 0, 0, 0);
    for (long long i = n4 * 4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        dense[i] = 0;
}

// One CTA per root with UB > CC_MAXUB: counts in a dense global row of n ints.
// Pass 1 adds every wedge; pass 2 reads each count (per middle vertex) and
// marks the key with the sign bit, so that exactly one visitor credits
// C(c, 2) to w; pass 3 stores zeros back.
__global__ void __launch_bounds__(CG_THREADS) k_c4_global(Graph g, VAcc *vacc, const int *lists, const int *counters,
                                                          int *dense, int slots) {
    constexpr int NW = CG_THREADS / 32;
    __shared__ __align__(8) int segs[NW][128];
    if ((int)blockIdx.x >= slots) return;
    int *row = dense + (size_t)blockIdx.x * g.n;
    const int wid = threadIdx.x >> 5, lane = lane_id();
    int *sst = segs[wid], *spre = sst + 32;
    long long *pv = reinterpret_cast<long long *>(spre + 32);
    const int *glob_list = lists + 4 * (size_t)g.n;
    const int nh = counters[CNT_C4_GLOBAL];
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int u = glob_list[h];
        const int4 ru = g.rinfo[u];
        const int b = ru.x, din = ru.y - ru.x;
        pv[lane] = 0;
        walk_wedges(g, u, b, din, wid, NW, sst, spre, [&](int, int w) { atomicAdd(&row[w], 1); }, [&](int) {});
        __syncthreads();
        long long su = 0;
        walk_wedges(g, u, b, din, wid, NW, sst, spre,
                    [&](int q, int w) {
                        const int old = atomicOr(&row[w], (int)0x80000000);
                        const int c = old & 0x7fffffff;
                        if (c > 1) atomicAdd((unsigned long long *)&pv[q], (unsigned long long)(c - 1));
                        if (old >= 0 && c >= 2) {   // first visitor of this key
                            su += c2(c);
                            add64(&vacc[w].C4, c2(c));
                        }
                    },
                    [&](int v) {
                        const long long x = pv[lane];
                        if (x) add64(&vacc[v].C4, x);
                        pv[lane] = 0;
                    });
        su = warp_sum(su);
        if (lane == 0 && su) add64(&vacc[u].C4, su);
        __syncthreads();
        walk_wedges(g, u, b, din, wid, NW, sst, spre, [&](int, int w) { row[w] = 0; }, [&](int) {});
        __syncthreads();
    }
}

void launch_cycle4(Work &w, cudaStream_t st) {
    Graph g{w.n, w.m, w.rinfo, w.ncol};
    const int maxub = w.tune[TUNE_C4_WARP_MAXW] < CW_MAXUB ? w.tune[TUNE_C4_WARP_MAXW] : CW_MAXUB;
    k_c4_warp<<<w.num_sms * w.tune[TUNE_GRID_C4], CW_WARPS * 32, 0, st>>>(g, w.vacc, w.lists, w.counters, maxub);
    after_launch(st, K_C4_WARP);
    k_c4_mid<<<w.num_sms * 4, CM_THREADS, CM_SMEM, st>>>(g, w.vacc, w.lists, w.counters);
    after_launch(st, K_C4_MID);
    k_c4_cta<<<w.num_sms, CC_THREADS, CC_SMEM, st>>>(g, w.vacc, w.lists, w.counters);
    after_launch(st, K_C4_CTA);
    if (w.c4slots > 0) {
        k_c4_zero_dense<<<w.num_sms * 4, 256, 0, st>>>(w.c4dense, w.n, w.c4slots, w.counters);
        after_launch(st, K_C4_ZERO);
        k_c4_global<<<w.c4slots, CG_THREADS, 0, st>>>(g, w.vacc, w.lists, w.counters, w.c4dense, w.c4slots);
        after_launch(st, K_C4_GLOBAL);
    }
}

void configure_cycle4() {
    cudaFuncSetAttribute(k_c4_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CM_SMEM);
    cudaFuncSetAttribute(k_c4_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC_SMEM);
}

}  // namespace niorca
