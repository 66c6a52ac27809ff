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
// With rows sorted, the wedges through v are the prefix of row v below u,
// cut by a binary search for u. Tiers by wedge count W(u): one warp with a
// 1024-slot shared table; one CTA with a 16384-slot shared table; one CTA
// with a dense count row in global memory for the largest roots.
#include "kernels.h"

namespace niorca {

constexpr int CW_WARPS = 4;   // 4 x 11 KB of static shared memory
constexpr int CW_SLOTS = 1024;
constexpr int CW_MAXW = CW_SLOTS / 2;
constexpr int CC_THREADS = 512;
constexpr int CC_SLOTS = 16384;
constexpr int CC_MAXW = CC_SLOTS / 2;
constexpr size_t CC_SMEM = (size_t)CC_SLOTS * 8 + (size_t)(CC_THREADS / 32) * 128 * 4;
constexpr int CG_THREADS = 1024;

__device__ __forceinline__ int seg_owner3(const int *pre, int k) {
    int lo = 0, hi = 31;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ long long c2(long long c) { return c * (c - 1) / 2; }

// Wedges through in-neighbour v of root u: row v from its start up to the
// position of u, which lies in v's out-part [rv.y, rv.z).
__device__ __forceinline__ int wedge_len(const Graph &g, int v, int u) {
    const int4 rv = g.rinfo[v];
    return lower_bound(g.ncol, rv.y, rv.z, u) - rv.x;
}

// Walks the wedges of root u: for every chunk of 32 in-neighbours (starting
// at chunk `c0`, step `cstep` chunks), sets up the segment table of the warp
// and calls f(q, pos) for each wedge (q: lane that owns v, pos: position of w),
// then done(v, seg_len) once per chunk after a __syncwarp. `lens`, when not
// null, holds the segment length of the first `nlens` in-neighbours.
template <class F, class D>
__device__ __forceinline__ void walk_wedges(const Graph &g, int u, int b, int din, int c0, int cstep, int *sst,
                                            int *spre, F f, D done, const int *lens = nullptr, int nlens = 0) {
    const int lane = lane_id();
    for (int cb = c0 * 32; cb < din; cb += cstep * 32) {
        const int p = cb + lane;
        int v = -1, st = 0, len = 0;
        if (p < din) {
            v = g.ncol[b + p];
            const int4 rv = g.rinfo[v];
            st = rv.x;
            len = p < nlens ? lens[p] : lower_bound(g.ncol, rv.y, rv.z, u) - rv.x;
        }
        const int incl = warp_inclusive_scan(len);
        sst[lane] = st;
        spre[lane] = incl - len;
        const int total = __shfl_sync(FULL, incl, 31);
        __syncwarp();
        for (int kb = 0; kb < total; kb += 32) {
            const int k = kb + lane;
            if (k >= total) break;
            const int q = seg_owner3(spre, k);
            f(q, sst[q] + (k - spre[q]));
        }
        __syncwarp();
        done(v, len);
        __syncwarp();
    }
}

constexpr int CW_LENS = 64;   // cached wedge-segment lengths per root

struct C4WarpSmem {
    int hk[CW_SLOTS];      // keys (-1 = empty); all empty between roots
    int hc[CW_SLOTS];      // wedge counts per key
    int touched[CW_MAXW];  // slots filled by the current root
    int lens[CW_LENS];
    int sst[32];
    int spre[32];
    long long pv[32];
    int ntouched;
};

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

// One warp per root with at most CW_MAXW wedges. The table is cleared once
// per warp; afterwards every root empties only the slots it filled.
__global__ void __launch_bounds__(CW_WARPS * 32) k_c4_warp(Graph g, VAcc *vacc, int *lists, int *counters,
                                                           int maxw) {
    __shared__ C4WarpSmem sm_all[CW_WARPS];
    C4WarpSmem &S = sm_all[threadIdx.x >> 5];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int *cta_list = lists + 2 * (size_t)g.n;
    int *glob_list = lists + 3 * (size_t)g.n;
    constexpr unsigned mask = CW_SLOTS - 1;
    for (int i = lane; i < CW_SLOTS; i += 32) { S.hk[i] = -1; S.hc[i] = 0; }
    if (lane == 0) S.ntouched = 0;
    __syncwarp();
    for (int u = gw; u < g.n; u += nw) {
        const int4 ru = g.rinfo[u];
        const int b = ru.x, din = ru.y - ru.x;
        if (din < 2) continue;
        long long W = 0;
        for (int p = lane; p < din; p += 32) {
            const int len = wedge_len(g, g.ncol[b + p], u);
            if (p < CW_LENS) S.lens[p] = len;
            W += len;
        }
        W = warp_sum(W);
        if (W < 2) continue;
        if (W > maxw) {
            if (lane == 0) {
                if (W > CC_MAXW) glob_list[atomicAdd(&counters[CNT_C4_GLOBAL], 1)] = u;
                else cta_list[atomicAdd(&counters[CNT_C4_CTA], 1)] = u;
            }
            continue;
        }
        __syncwarp();
        walk_wedges(
            g, u, b, din, 0, 1, S.sst, S.spre,
            [&](int, int pos) {
                const int slot = hcount_add_new(S.hk, S.hc, mask, g.ncol[pos]);
                if (slot >= 0) S.touched[atomicAdd(&S.ntouched, 1)] = slot;
            },
            [&](int, int) {}, S.lens, CW_LENS);
        const int nt = S.ntouched;
        long long su = 0;
        for (int i = lane; i < nt; i += 32) {
            const int slot = S.touched[i];
            const int c = S.hc[slot];
            if (c >= 2) {
                su += c2(c);
                add64(&vacc[S.hk[slot]].C4, c2(c));
            }
        }
        su = warp_sum(su);
        if (lane == 0 && su) add64(&vacc[u].C4, su);
        if (su) {   // middle vertices, only when some cycle is rooted at u
            S.pv[lane] = 0;
            __syncwarp();
            walk_wedges(
                g, u, b, din, 0, 1, S.sst, S.spre,
                [&](int q, int pos) {
                    const int c = hcount_get(S.hk, S.hc, mask, g.ncol[pos]);
                    if (c > 1) atomicAdd((unsigned long long *)&S.pv[q], (unsigned long long)(c - 1));
                },
                [&](int v, int) {
                    const long long x = S.pv[lane];
                    if (x) add64(&vacc[v].C4, x);
                    S.pv[lane] = 0;
                },
                S.lens, CW_LENS);
        }
        for (int i = lane; i < nt; i += 32) {
            const int slot = S.touched[i];
            S.hk[slot] = -1;
            S.hc[slot] = 0;
        }
        __syncwarp();
        if (lane == 0) S.ntouched = 0;
        __syncwarp();
    }
}

// One CTA per root with CW_MAXW < W <= CC_MAXW: the table in shared memory.
__global__ void __launch_bounds__(CC_THREADS) k_c4_cta(Graph g, VAcc *vacc, const int *lists, const int *counters) {
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int NW = CC_THREADS / 32;
    int *hk = reinterpret_cast<int *>(dsm);
    int *hc = hk + CC_SLOTS;
    const int wid = threadIdx.x >> 5, lane = lane_id();
    int *sst = hc + CC_SLOTS + wid * 128;
    int *spre = sst + 32;
    long long *pv = reinterpret_cast<long long *>(spre + 32);
    const int *cta_list = lists + 2 * (size_t)g.n;
    const int nh = counters[CNT_C4_CTA];
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int u = cta_list[h];
        const int4 ru = g.rinfo[u];
        const int b = ru.x, din = ru.y - ru.x;
        for (int i = threadIdx.x; i < CC_SLOTS; i += CC_THREADS) { hk[i] = -1; hc[i] = 0; }
        pv[lane] = 0;
        __syncthreads();
        const unsigned mask = CC_SLOTS - 1;
        walk_wedges(g, u, b, din, wid, NW, sst, spre,
                    [&](int, int pos) { hcount_add(hk, hc, mask, g.ncol[pos]); }, [&](int, int) {});
        __syncthreads();
        long long su = 0;
        for (int i = threadIdx.x; i < CC_SLOTS; i += CC_THREADS) {
            const int c = hc[i];
            if (c >= 2) {
                su += c2(c);
                add64(&vacc[hk[i]].C4, c2(c));
            }
        }
        su = warp_sum(su);
        if (lane == 0 && su) add64(&vacc[u].C4, su);
        walk_wedges(g, u, b, din, wid, NW, sst, spre,
                    [&](int q, int pos) {
                        const int c = hcount_get(hk, hc, mask, g.ncol[pos]);
                        if (c > 1) atomicAdd((unsigned long long *)&pv[q], (unsigned long long)(c - 1));
                    },
                    [&](int v, int) {
                        const long long x = pv[lane];
                        if (x) add64(&vacc[v].C4, x);
                        pv[lane] = 0;
                    });
        __syncthreads();
    }
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

// One CTA per root with W > CC_MAXW: counts in a dense global row of n ints,
// which the third pass returns to zero.
__global__ void __launch_bounds__(CG_THREADS) k_c4_global(Graph g, VAcc *vacc, const int *lists, const int *counters,
                                                          int *dense, int slots) {
    constexpr int NW = CG_THREADS / 32;
    __shared__ __align__(8) int segs[NW][128];
    if ((int)blockIdx.x >= slots) return;
    int *row = dense + (size_t)blockIdx.x * g.n;
    const int wid = threadIdx.x >> 5, lane = lane_id();
    int *sst = segs[wid], *spre = sst + 32;
    long long *pv = reinterpret_cast<long long *>(spre + 32);
    const int *glob_list = lists + 3 * (size_t)g.n;
    const int nh = counters[CNT_C4_GLOBAL];
    for (int h = blockIdx.x; h < nh; h += gridDim.x) {
        const int u = glob_list[h];
        const int4 ru = g.rinfo[u];
        const int b = ru.x, din = ru.y - ru.x;
        pv[lane] = 0;
        walk_wedges(g, u, b, din, wid, NW, sst, spre, [&](int, int pos) { atomicAdd(&row[g.ncol[pos]], 1); },
                    [&](int, int) {});
        __syncthreads();
        walk_wedges(g, u, b, din, wid, NW, sst, spre,
                    [&](int q, int pos) {
                        const int c = __ldcg(&row[g.ncol[pos]]);   // counts were added at L2
                        if (c > 1) atomicAdd((unsigned long long *)&pv[q], (unsigned long long)(c - 1));
                    },
                    [&](int v, int) {
                        const long long x = pv[lane];
                        if (x) add64(&vacc[v].C4, x);
                        pv[lane] = 0;
                    });
        __syncthreads();
        long long su = 0;
        walk_wedges(g, u, b, din, wid, NW, sst, spre,
                    [&](int, int pos) {
                        const int w = g.ncol[pos];
                        const int c = atomicExch(&row[w], 0);
                        if (c >= 2) {
                            su += c2(c);
                            add64(&vacc[w].C4, c2(c));
                        }
                    },
                    [&](int, int) {});
        su = warp_sum(su);
        if (lane == 0 && su) add64(&vacc[u].C4, su);
        __syncthreads();
    }
}

void launch_cycle4(Work &w, cudaStream_t st) {
    Graph g{w.n, w.m, w.rinfo, w.ncol};
    const int maxw = w.tune[TUNE_C4_WARP_MAXW] < CW_MAXW ? w.tune[TUNE_C4_WARP_MAXW] : CW_MAXW;
    k_c4_warp<<<w.num_sms * w.tune[TUNE_GRID_C4], CW_WARPS * 32, 0, st>>>(g, w.vacc, w.lists, w.counters, maxw);
    after_launch(st, K_C4_WARP);
    k_c4_cta<<<w.num_sms * 2, CC_THREADS, CC_SMEM, st>>>(g, w.vacc, w.lists, w.counters);
    after_launch(st, K_C4_CTA);
    if (w.c4slots > 0) {
        k_c4_zero_dense<<<w.num_sms * 4, 256, 0, st>>>(w.c4dense, w.n, w.c4slots, w.counters);
        after_launch(st, K_C4_ZERO);
        k_c4_global<<<w.c4slots, CG_THREADS, 0, st>>>(g, w.vacc, w.lists, w.counters, w.c4dense, w.c4slots);
        after_launch(st, K_C4_GLOBAL);
    }
}

void configure_cycle4() {
    cudaFuncSetAttribute(k_c4_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC_SMEM);
}

}  // namespace niorca
