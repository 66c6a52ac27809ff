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
// The wedges through v are the entries of row v below u: a prefix of row v
// ending at the position of u, which a search of N+(v) finds. Roots are
// routed by their wedge count W (a count is at most W too): one warp with a
// 6 KB table (k_c4_warp) or an 8 KB one (k_c4_warp_big), four warps
// (k_c4_mid, packed or split tables), a 512-thread CTA (k_c4_cta), or, for the largest
// roots, and for every root with more than WL_MAXD in-neighbours, a
// 1024-thread CTA that counts the root's key range tile by tile in shared
// memory (k_c4_tiled). The other tables are open-addressing hash
// tables in shared memory, either split (key and count arrays) or packed
// (key << cb | count in one 32-bit word, cb = 32 - bits(n - 1) count bits,
// usable while W < 2^cb - 1), which holds twice the keys in the same space.
// Each table is emptied once per CTA; afterwards a warp sweeps the region
// its root used, and a CTA empties the slots it filled (kept in a 16-bit
// `touched` list).
#include "kernels.h"

namespace niorca {

constexpr int CW_WARPS = 4;
constexpr int CW_WORDS = 1536;      // table words per warp of k_c4_warp: 6 KB, 8 CTAs of 4 warps per SM
constexpr int CWB_WORDS = 2048;     // k_c4_warp_big: 8 KB, 6 CTAs per SM
constexpr int CW_MAXW = 1536;       // largest W of a root in the warp tiers
constexpr int CW_SMALL_MAXW = 256;  // the same, for graphs with fewer vertices than resident warps
constexpr int CW_DUPS = 32;         // repeated keys a warp credits by search at most
constexpr int CW_BIG_LIST = 0;      // list slot of k_c4_warp_big's roots: the triangle stage's heavy list,
                                    // which nothing reads after that stage
constexpr int CM_THREADS = 128;
constexpr int CM_SLOTS = 4096;      // split; 8192 when packed
constexpr int CM_MAXW = 3072;      // split; 6144 when packed
constexpr int CC_THREADS = 512;
constexpr int CC_SLOTS = 16384;     // split
constexpr int CC_MAXW = 12288;
constexpr unsigned EMPTY = 0xffffffffu;

__device__ __forceinline__ long long c2(long long c) { return c * (c - 1) / 2; }

// Adds c - 1 to pv[q] (shared) for the lanes with c > 1; lanes of one
// in-neighbour q are consecutive in a window, so one add per run. A window
// that lies inside one in-neighbour's run (the usual case on long rows)
// takes one warp reduction and one add.
__device__ __forceinline__ void add_middle(long long *pv, int q, int c) {
    const unsigned v = c > 1 ? (unsigned)(c - 1) : 0u;
    if (!__any_sync(FULL, v != 0)) return;
    const int q0 = __shfl_sync(FULL, q, 0);
    if (__all_sync(FULL, q == q0 || v == 0)) {
        const unsigned t = __reduce_add_sync(FULL, v);
        if (lane_id() == 0) atomicAdd(reinterpret_cast<unsigned long long *>(&pv[q0]), (unsigned long long)t);
        return;
    }
    run_add(&pv[q], q, v);
}

// Wedges u - v - w through the in-neighbour v of root u: the entries of row
// v below u, i.e. the position of u in row v (u is in N+(v)), found by a
// search of N+(v) whose last steps touch the lines the walk reads next.
__device__ __forceinline__ int wedge_len(const Graph &g, int u, const int4 &rv) {
    return lower_bound(g.ncol, rv.y, rv.z, u) - rv.x;
}

// The wedge segment {row start, length} of the in-neighbour at position p of
// row u (din = u's in-degree): from the table k_c4_wedge_len filled, for the
// rows it covers, else by a search of N+(v).
__device__ __forceinline__ int2 wedge_seg(const Graph &g, int u, int din, int p) {
    if (din <= WL_MAXD) return g.wl[p];
    const int4 rv = g.rinfo[g.ncol[p]];
    return make_int2(rv.x, wedge_len(g, u, rv));
}

// The wedge segment of every in-entry of the rows with at most WL_MAXD
// in-neighbours, a group of L lanes per row (16, or 8 for graphs of mean
// degree below 16): the row gather and binary search of each entry, made
// here with every thread independent, so that the per-root kernels read one
// coalesced 8-byte entry per in-neighbour.
template <int L>
__global__ void __launch_bounds__(256, 8) k_c4_wedge_len(Graph g, int2 *wl, const int *counters) {
    pdl_begin();
    if (degree_overflow(counters)) return;
    const int hl = threadIdx.x & (L - 1);
    const int gh = (blockIdx.x * blockDim.x + threadIdx.x) / L, nh = (gridDim.x * blockDim.x) / L;
    for (int u = gh; u < g.n; u += nh) {
        const int4 ru = g.rinfo[u];
        if (ru.y - ru.x > WL_MAXD) continue;
        for (int p = ru.x + hl; p < ru.y; p += L) {
            const int4 rv = g.rinfo[g.ncol[p]];
            wl[p] = make_int2(rv.x, wedge_len(g, u, rv));
        }
    }
}

// Segment table of in-neighbour chunk cb of root u in the calling warp: the
// wedge prefixes of the rows of v = ncol[b + cb + lane] concatenated. Returns
// the total length; the lane's own v, segment length and offset come back in
// v, len, pre.
__device__ __forceinline__ int wedge_chunk(const Graph &g, int u, int b, int din, int cb, SegTab &T, int &v,
                                           int &len, int &pre) {
    const int p = cb + lane_id();
    int st = 0;
    v = -1;
    len = 0;
    if (p < din) {
        v = g.ncol[b + p];
        const int2 sl = wedge_seg(g, u, din, b + p);
        st = sl.x;
        len = sl.y;
    }
    return seg_build(T, st, len, pre);
}

// Wedge segments of a root's first two chunks of in-neighbours, held in
// registers by the warp (lane p: in-neighbours p and 32 + p) so that its
// walks search no row again. With one chunk (din <= 32) its segment table
// may be built already (built0: pre0 and total0 are the lane's).
struct RootChunks {
    int have = 0;          // chunks held: 0, 1 or 2 (warp-uniform)
    bool built0 = false;   // the warp's segment table holds chunk 0
    int v0 = -1, st0 = 0, len0 = 0, v1 = -1, st1 = 0, len1 = 0;
    int pre0 = 0, total0 = 0;
};

// Segment table of chunk c (in-neighbours 32c ...) of root u, from the
// registers of rc when it holds the chunk, else by searching the rows.
__device__ __forceinline__ int root_chunk(const Graph &g, int u, int b, int din, int c, SegTab &T,
                                          const RootChunks &rc, int &v, int &len, int &pre) {
    if (c == 0 && rc.built0) {
        v = rc.v0, len = rc.len0, pre = rc.pre0;
        return rc.total0;
    }
    if (c < rc.have) {
        v = c == 0 ? rc.v0 : rc.v1;
        len = c == 0 ? rc.len0 : rc.len1;
        return seg_build(T, c == 0 ? rc.st0 : rc.st1, len, pre);
    }
    return wedge_chunk(g, u, b, din, 32 * c, T, v, len, pre);
}

// Walks the wedges of root u (in-neighbours b .. b + din of row u) in the
// calling warp, chunk by chunk of 32 in-neighbours: f(act, q, w) on every
// lane, act meaning that w is a wedge end through the v owned by lane q;
// then done(v) per chunk.
template <class F, class D>
__device__ __forceinline__ void walk_wedges(const Graph &g, int u, int b, int din, SegTab &T, F f, D done,
                                            const RootChunks &rc) {
    for (int c = 0; 32 * c < din; ++c) {
        int v, len, pre;
        const int total = root_chunk(g, u, b, din, c, T, rc, v, len, pre);
        seg_visit32<4>(g.ncol, T, pre, len, total, 0, [&](bool ok, int q, int, int w) { f(ok, q, w); });
        __syncwarp();
        done(v);
        __syncwarp();
    }
}

// The same walk shared by all warps of a CTA: every warp builds the segment
// table of each chunk and takes the windows wid, wid + nw, ... of 32
// elements. With DONE, warp 0 calls done(v) after the CTA finished the chunk.
template <bool DONE, class F, class D>
__device__ __forceinline__ void walk_wedges_cta(const Graph &g, int u, int b, int din, int wid, int nw,
                                                SegTab &T, F f, D done) {
    for (int cb = 0; cb < din; cb += 32) {
        int v, len, pre;
        const int total = wedge_chunk(g, u, b, din, cb, T, v, len, pre);
        seg_visit<4>(g.ncol, T, pre, len, total, wid * 32, nw * 32, [&](bool ok, int q, int, int w) { f(ok, q, w); });
        if (DONE) {
            __syncthreads();
            if (wid == 0) done(v);
            __syncthreads();
        } else {
            __syncwarp();
        }
    }
}

// Probe sequence of the 4-cycle count tables (any size S): first the high
// word of S times the key times 2^32 / golden ratio (Fibonacci hashing; for
// S = 2^k the top k bits of the product), then the same with a second
// multiplier, then linear from there. Keys whose first slots collide part
// ways at the second probe, which keeps the runs, and so a warp's slowest
// insert, short.
__device__ __forceinline__ unsigned fib_slot(int key, unsigned size) {
    return __umulhi(static_cast<unsigned>(key) * 0x9E3779B1u, size);
}
__device__ __forceinline__ unsigned next_probe(unsigned s, unsigned probe, int key, unsigned size) {
    return probe == 0 ? __umulhi(static_cast<unsigned>(key) * 0x85EBCA77u, size) : (s + 1 == size ? 0u : s + 1);
}

// Split table of `size` slots: keys (-1 empty) and counts in two arrays.
struct SplitTab {
    int *hk, *hc;
    unsigned size;
    unsigned short *touched;   // slots filled (CTA groups)
    // counts w; returns the slot if this call inserted w, -1 if w was there
    __device__ __forceinline__ int add(int w) const {
        unsigned s = fib_slot(w, size);
        for (unsigned probe = 0; probe < size; ++probe) {
            const int prev = atomicCAS(&hk[s], -1, w);
            if (prev == -1) { atomicAdd(&hc[s], 1); return (int)s; }
            if (prev == w) { atomicAdd(&hc[s], 1); return -1; }
            s = next_probe(s, probe, w, size);
        }
        return -1;
    }
    // Counts w (warp tier); true for the one call whose increment takes
    // w's count from 1 to 2, so that each repeated key is reported once.
    __device__ __forceinline__ bool add_rep(int w) const {
        unsigned s = fib_slot(w, size);
        for (unsigned probe = 0; probe < size; ++probe) {
            const int prev = atomicCAS(&hk[s], -1, w);
            if (prev == -1 || prev == w) return atomicAdd(&hc[s], 1) == 1;
            s = next_probe(s, probe, w, size);
        }
        return false;
    }
    __device__ __forceinline__ int get(int w) const {
        unsigned s = fib_slot(w, size);
        for (unsigned probe = 0; probe < size; ++probe) {
            const int k = hk[s];
            if (k == w) return hc[s];
            if (k == -1) return 0;
            s = next_probe(s, probe, w, size);
        }
        return 0;
    }
    __device__ __forceinline__ bool empty(int s) const { return hk[s] == -1; }
    __device__ __forceinline__ int key(int s) const { return hk[s]; }
    __device__ __forceinline__ int cnt(int s) const { return hc[s]; }
    __device__ __forceinline__ void clear(int s) const { hk[s] = -1; hc[s] = 0; }
    __device__ __forceinline__ void clear_all(int tid, int nthreads) const {
        for (int i = tid; i < (int)size; i += nthreads) { hk[i] = -1; hc[i] = 0; }
    }
};

// Packed table of `size` slots (a multiple of 4): one word (w << cb) |
// count per slot, EMPTY when free. A count never reaches 2^cb - 1 (the
// caller ensures W < 2^cb - 1), so a full word is never EMPTY.
struct PackedTab {
    unsigned *t;
    unsigned size;
    int cb;
    unsigned short *touched;   // slots filled (CTA groups)
    __device__ __forceinline__ int add(int w) const {
        const unsigned key = static_cast<unsigned>(w);
        unsigned s = fib_slot(w, size);
        for (unsigned probe = 0; probe < size; ++probe) {
            const unsigned prev = atomicCAS(&t[s], EMPTY, (key << cb) | 1u);
            if (prev == EMPTY) return (int)s;
            if ((prev >> cb) == key) { atomicAdd(&t[s], 1u); return -1; }
            s = next_probe(s, probe, w, size);
        }
        return -1;
    }
    __device__ __forceinline__ bool add_rep(int w) const {
        const unsigned key = static_cast<unsigned>(w);
        unsigned s = fib_slot(w, size);
        for (unsigned probe = 0; probe < size; ++probe) {
            const unsigned prev = atomicCAS(&t[s], EMPTY, (key << cb) | 1u);
            if (prev == EMPTY) return false;
            if ((prev >> cb) == key) return (atomicAdd(&t[s], 1u) & ((1u << cb) - 1)) == 1;
            s = next_probe(s, probe, w, size);
        }
        return false;
    }
    __device__ __forceinline__ int get(int w) const {
        const unsigned key = static_cast<unsigned>(w);
        unsigned s = fib_slot(w, size);
        for (unsigned probe = 0; probe < size; ++probe) {
            const unsigned cur = t[s];
            if (cur == EMPTY) return 0;
            if ((cur >> cb) == key) return (int)(cur & ((1u << cb) - 1));
            s = next_probe(s, probe, w, size);
        }
        return 0;
    }
    __device__ __forceinline__ bool empty(int s) const { return t[s] == EMPTY; }
    __device__ __forceinline__ int key(int s) const { return (int)(t[s] >> cb); }
    __device__ __forceinline__ int cnt(int s) const { return (int)(t[s] & ((1u << cb) - 1)); }
    __device__ __forceinline__ void clear(int s) const { t[s] = EMPTY; }
    __device__ __forceinline__ void clear_all(int tid, int nthreads) const {
        uint4 *t4 = reinterpret_cast<uint4 *>(t);
        for (int i = tid; i < (int)size / 4; i += nthreads) t4[i] = make_uint4(EMPTY, EMPTY, EMPTY, EMPTY);
    }
};

// Counts all wedges of u into the table and credits every 4-cycle rooted at
// u. Every thread of the group (one warp, or a CTA with CTA = true) calls it.
// A repeated key is a 4-cycle, so roots without one skip the credit and
// middle passes. A CTA records the slots it fills in `touched` (flags[0]
// counts them, flags[1] notes a repeated key) and empties only those; a warp
// keeps no list of slots: it uses its whole table for every root, clears all
// of it, and has each repeated key reported by the insert that makes its
// count 2.
// pv holds the per-middle-vertex sums of one chunk (per warp, or shared by
// the CTA).
template <bool CTA, class Tab>
__device__ __forceinline__ void c4_root(const Graph &g, VAcc *vacc, int u, int b, int din,
                                        const Tab &T, int wid, int nw, int tid, int nthreads, SegTab &seg,
                                        long long *pv, int *flags, const RootChunks &rc = RootChunks{},
                                        long long W = 0) {
    const int lane = lane_id();
    auto sync = [] {
        if (CTA) __syncthreads(); else __syncwarp();
    };
    int nrep = 0;   // warp group: repeated keys, the first CW_DUPS of them listed in flags[]
    auto insert = [&](bool act, int, int w) {
        if (!CTA) {
            const bool rep = act && T.add_rep(w);
            const unsigned r = __ballot_sync(FULL, rep);
            if (r) {
                const int at = nrep + __popc(r & lanemask_lt());
                if (rep && at < CW_DUPS) flags[at] = w;
                nrep += __popc(r);
            }
            return;
        }
        const int slot = act ? T.add(w) : -2;
        // new keys of the warp take consecutive `touched` entries
        const unsigned fresh = __ballot_sync(FULL, slot >= 0);
        const unsigned dups = __ballot_sync(FULL, slot == -1);
        if (!(fresh | dups)) return;
        int base = 0;
        if (fresh && lane == __ffs(fresh) - 1) base = atomicAdd(&flags[0], __popc(fresh));
        if (dups && lane == 0) flags[1] = 1;
        if (slot >= 0) {
            base = __shfl_sync(fresh, base, __ffs(fresh) - 1);
            T.touched[base + __popc(fresh & lanemask_lt())] = (unsigned short)slot;
        }
    };
    if (CTA) walk_wedges_cta<false>(g, u, b, din, wid, nw, seg, insert, [](int) {});
    else walk_wedges(g, u, b, din, seg, insert, [](int) {}, rc);
    sync();
    const int nt = CTA ? flags[0] : (int)T.size;   // entries of the list, or slots swept
    bool sweep = CTA ? flags[1] != 0 : false;
    if (!CTA && nrep > 0) {
        // The repeated keys (count >= 2) of a warp's root were reported once
        // each during the walk; up to CW_DUPS of them are listed in flags[],
        // which gives their final counts without sweeping the table (more:
        // a sweep). Each is credited C(c, 2); the middle vertices of key w
        // are N-(u) ∩ N(w), found by searching row w for each in-neighbour
        // (one search per lane and pair), while the pairs number at most
        // W / 4: each search is a short chain of dependent loads, and a root
        // of a small dense graph with tens of repeated keys walks its few
        // windows again sooner. Otherwise: the middle walk below.
        long long su = 0;
        const int nd = nrep;
        if (nd <= CW_DUPS) {
            for (int k = lane; k < nd; k += 32) {
                const int w = flags[k], c = T.get(w);
                flags[CW_DUPS + k] = c;
                su += c2(c);
                add64(&vacc[w].C4, c2(c));
            }
        } else {
            for (int i = lane; i < nt; i += 32) {
                if (T.empty(i)) continue;
                const int c = T.cnt(i);
                if (c >= 2) {
                    su += c2(c);
                    add64(&vacc[T.key(i)].C4, c2(c));
                }
            }
        }
        su = warp_sum(su);
        if (lane == 0) add64(&vacc[u].C4, su);
        __syncwarp();
        if (nd <= CW_DUPS && (long long)nd * din * 4 <= W) {
            // one (key, in-neighbour) pair per lane, all searches independent
            for (int t = lane; t < nd * din; t += 32) {
                const int k = t / din, p = t - k * din;
                const int w = flags[k], c = flags[CW_DUPS + k];
                const int4 rw = g.rinfo[w];
                const int v = g.ncol[b + p];
                if (find_sorted(g.ncol, rw.x, rw.z, v) >= 0) add64(&vacc[v].C4, c - 1);
            }
            __syncwarp();
        } else {
            sweep = true;   // credits done; middle walk only
        }
    }
    if (sweep) {
        long long su = 0;
        for (int i = tid; i < (CTA ? nt : 0); i += nthreads) {
            const int slot = CTA ? T.touched[i] : i;
            if (!CTA && T.empty(slot)) continue;
            const int c = T.cnt(slot);
            if (c >= 2) {
                su += c2(c);
                add64(&vacc[T.key(slot)].C4, c2(c));
            }
        }
        su = warp_sum(su);
        if (CTA && lane == 0 && su) add64(&vacc[u].C4, su);
        // middle vertices: each wedge through v adds c_w - 1
        if (tid < 32) pv[tid] = 0;
        sync();
        auto middle = [&](bool act, int q, int w) {   // lanes of one v add once
            const int c = act ? T.get(w) : 0;
            add_middle(pv, q, c);
        };
        auto flush = [&](int v) {
            const long long x = pv[lane];
            if (x) add64(&vacc[v].C4, x);
            pv[lane] = 0;
        };
        if (CTA) walk_wedges_cta<true>(g, u, b, din, wid, nw, seg, middle, flush);
        else walk_wedges(g, u, b, din, seg, middle, flush, rc);
        sync();
    }
    if (CTA) {
        for (int i = tid; i < nt; i += nthreads) T.clear(T.touched[i]);
        sync();
        if (tid == 0) {
            flags[0] = 0;
            flags[1] = 0;
        }
    } else {
        T.clear_all(tid, nthreads);
    }
    sync();
}


template <int WORDS>
struct __align__(16) C4WarpSmem {
    unsigned t[WORDS];
    SegTab seg;
    long long pv[32];
    int dups[2 * CW_DUPS];   // repeated keys of a root and their counts
};

// Slots of a warp's table of WORDS words (packed words, or split (key,
// count) pairs), and the largest W it takes: 3/4 of the slots.
__host__ __device__ constexpr int cw_slots(bool split, int words) { return split ? words / 2 : words; }
__host__ __device__ constexpr int cw_maxw(bool split, int words) { return cw_slots(split, words) / 4 * 3; }

// One warp per root. k_c4_warp (BIG = false) takes every vertex as a root:
// those with W up to 3/4 of its 6 KB table are counted there, those that
// fit the 8 KB table of k_c4_warp_big (BIG = true) are queued for it, the
// rest for the wider tiers. SPLIT: (key, count) pair tables, for graphs
// whose ids leave a packed word too few count bits.
template <bool SPLIT, bool BIG>
__device__ __forceinline__ void c4_warp_body(Graph g, VAcc *vacc, int *lists, int *counters, int maxw, int cb,
                                             int teamw) {
    if (degree_overflow(counters)) return;
    constexpr int WORDS = BIG ? CWB_WORDS : CW_WORDS;
    constexpr int TS = cw_slots(SPLIT, WORDS);
    __shared__ C4WarpSmem<WORDS> sm_all[CW_WARPS];
    C4WarpSmem<WORDS> &S = sm_all[threadIdx.x >> 5];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const long long pack_lim = (1ll << cb) - 2;   // largest W a packed count may reach
    const long long warp_cap = SPLIT ? maxw : (maxw < pack_lim ? maxw : pack_lim);   // W the warp tiers take
    const long long here_lim = warp_cap < cw_maxw(SPLIT, WORDS) ? warp_cap : cw_maxw(SPLIT, WORDS);
    const long long big_lim = warp_cap < cw_maxw(SPLIT, CWB_WORDS) ? warp_cap : cw_maxw(SPLIT, CWB_WORDS);
    int *const big_roots = lists + (size_t)CW_BIG_LIST * g.n;
    const int count = BIG ? counters[CNT_C4_WBIG] : g.n;
    auto root = [&](int i) { return BIG ? big_roots[i] : i; };
    int *const sk = reinterpret_cast<int *>(S.t), *const sc = sk + TS;   // split keys, counts
    if (SPLIT) SplitTab{sk, sc, (unsigned)TS, nullptr}.clear_all(lane, 32);
    else PackedTab{S.t, (unsigned)TS, cb, nullptr}.clear_all(lane, 32);
    __syncwarp();
    // Software pipeline over the warp's roots i, i + nw, i + 2 nw: row bounds
    // are loaded two roots ahead, the first 32 in-neighbours and their row
    // bounds one root ahead, so that a root starts with its data in flight.
    const int4 Z = make_int4(0, 0, 0, 0);
    int i = gw;
    int u = i < count ? root(i) : 0;
    int un = i + nw < count ? root(i + nw) : 0;
    int4 ru = i < count ? g.rinfo[u] : Z;
    int4 ru1 = i + nw < count ? g.rinfo[un] : Z;
    const int2 Z2 = make_int2(0, 0);
    // wedge segment through in-neighbour `lane` of the current root
    int2 s0 = (i < count && lane < ru.y - ru.x && ru.y - ru.x <= 64) ? g.wl[ru.x + lane] : Z2;
    for (; i < count; i += nw) {
        const int i2 = i + 2 * nw;
        const int u2 = i2 < count ? root(i2) : 0;
        const int4 ru2 = i2 < count ? g.rinfo[u2] : Z;
        const int2 s1 = (i + nw < count && lane < ru1.y - ru1.x && ru1.y - ru1.x <= 64) ? g.wl[ru1.x + lane] : Z2;
        [&] {
            const int b = ru.x, din = ru.y - ru.x;
            if (din < 2) return;
            long long W = 0;   // exact wedge count W of root u
            RootChunks rc;
            if (din <= 64) {   // both chunks' segments stay in registers
                rc.v0 = lane < din ? g.ncol[b + lane] : -1;   // for the middle walk's credits
                rc.st0 = s0.x;
                rc.len0 = s0.y;
                if (din <= 32) {   // one chunk: its segment table gives W
                    rc.have = 1;
                    rc.total0 = seg_build(S.seg, rc.st0, rc.len0, rc.pre0);
                    rc.built0 = true;
                    W = rc.total0;
                } else {
                    rc.have = 2;
                    if (32 + lane < din) {
                        rc.v1 = g.ncol[b + 32 + lane];
                        const int2 sl = g.wl[b + 32 + lane];
                        rc.st1 = sl.x;
                        rc.len1 = sl.y;
                    }
                    W = warp_sum(rc.len0 + rc.len1);
                }
            } else if (din <= WL_MAXD) {
                for (int p = lane; p < din; p += 32) W += g.wl[b + p].y;
                W = warp_sum(W);
            } else {
                // more in-neighbours than the wedge-segment table covers: the
                // key-tiled tier, which takes any root, without searching every
                // row for W here (one warp for a hub's rows would be the
                // kernel's tail); its order takes the in-neighbours' degree
                // sum, at least W, in W's place
#pragma unroll 8
                for (int p = lane; p < din; p += 32) {
                    const int4 rv = g.rinfo[g.ncol[b + p]];
                    W += rv.z - rv.x;
                }
                W = warp_sum(W);
            }
            const bool hub = din > WL_MAXD;
            if (W < 2 && !hub) return;
            if (W > here_lim || hub) {
                if (lane == 0) {
                    int which, list;   // queue counter and list slot (lists + list * n)
                    if (hub) { which = CNT_C4_TEAM; list = 4; }
                    else if (!BIG && W <= big_lim) { which = CNT_C4_WBIG; list = CW_BIG_LIST; }
                    else if (W > teamw) { which = CNT_C4_TEAM; list = 4; }
                    else if (W <= 2 * CM_MAXW && W <= pack_lim) { which = CNT_C4_MIDP; list = 5; }
                    else if (W <= CM_MAXW) { which = CNT_C4_MID; list = 2; }
                    else { which = CNT_C4_CTA; list = 3; }
                    const int at = atomicAdd(&counters[which], 1);
                    lists[(size_t)list * g.n + at] = u;
                    if (which == CNT_C4_TEAM)   // the order of the key-tiled tier
                        lists[(size_t)g.n + at] = (int)(W < 0x7fffffffll ? W : 0x7fffffffll);
                }
                return;
            }
            // every root takes the whole table: at the low load this leaves
            // (W / 1536 on the 6 KB table, about 0.2 on ER n = 1e6) a warp's
            // slowest insert needs fewer probes, which paid more (k_c4_warp
            // 1.58 -> 1.35 ms there) than the larger clear and sweep cost
            const unsigned slots = (unsigned)TS;
            if constexpr (SPLIT) {
                const SplitTab T{sk, sc, slots, nullptr};
                c4_root<false>(g, vacc, u, b, din, T, 0, 1, lane, 32, S.seg, S.pv, S.dups, rc, W);
            } else {
                const PackedTab T{S.t, slots, cb, nullptr};
                c4_root<false>(g, vacc, u, b, din, T, 0, 1, lane, 32, S.seg, S.pv, S.dups, rc, W);
            }
        }();
        u = un;
        un = u2;
        ru = ru1;
        ru1 = ru2;
        s0 = s1;
    }
}

// 8 CTAs of 4 warps per SM: 6 KB tables and at most 64 registers a thread.
__global__ void __launch_bounds__(CW_WARPS * 32, 8) k_c4_warp(Graph g, VAcc *vacc, int *lists, int *counters,
                                                              int maxw, int cb, int teamw) {
    pdl_begin();
    c4_warp_body<false, false>(g, vacc, lists, counters, maxw, cb, teamw);
}

__global__ void __launch_bounds__(CW_WARPS * 32, 8) k_c4_warp_split(Graph g, VAcc *vacc, int *lists,
                                                                    int *counters, int maxw, int cb, int teamw) {
    pdl_begin();
    c4_warp_body<true, false>(g, vacc, lists, counters, maxw, cb, teamw);
}

__global__ void __launch_bounds__(CW_WARPS * 32) k_c4_warp_big(Graph g, VAcc *vacc, int *lists, int *counters,
                                                               int maxw, int cb, int teamw) {
    pdl_begin();
    c4_warp_body<false, true>(g, vacc, lists, counters, maxw, cb, teamw);
}

__global__ void __launch_bounds__(CW_WARPS * 32) k_c4_warp_big_split(Graph g, VAcc *vacc, int *lists,
                                                                     int *counters, int maxw, int cb, int teamw) {
    pdl_begin();
    c4_warp_body<true, true>(g, vacc, lists, counters, maxw, cb, teamw);
}

// Roots from a queue, one CTA each. The table (SLOTS split slots, or
// 2 x SLOTS packed ones) lives in dynamic shared memory and is emptied once
// per CTA.
template <int THREADS, int SLOTS, int MAXW, bool PACKED>
__device__ __forceinline__ void c4_queue(const Graph &g, VAcc *vacc, const int *list, int count, int *next,
                                         int cb) {
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int NW = THREADS / 32;
    constexpr int NT = PACKED ? 2 * MAXW : MAXW;   // touched capacity: every key of a root
    unsigned *words = reinterpret_cast<unsigned *>(dsm);            // 2 x SLOTS words
    unsigned short *touched = reinterpret_cast<unsigned short *>(words + 2 * SLOTS);
    SegTab *segs = reinterpret_cast<SegTab *>(touched + NT);         // one per warp
    long long *pv = reinterpret_cast<long long *>(segs + NW);        // 32, shared by the CTA
    int *flags = reinterpret_cast<int *>(pv + 32);                  // new keys, repeated key
    const int wid = threadIdx.x >> 5;
    SegTab &seg = segs[wid];
    if (PACKED) {
        for (int i = threadIdx.x; i < 2 * SLOTS; i += THREADS) words[i] = EMPTY;
    } else {
        for (int i = threadIdx.x; i < SLOTS; i += THREADS) { words[i] = EMPTY; words[SLOTS + i] = 0; }
    }
    if (threadIdx.x == 0) { flags[0] = 0; flags[1] = 0; }
    __syncthreads();
    for (int h = cta_next(next); h < count; h = cta_next(next)) {
        const int u = list[h];
        const int4 ru = g.rinfo[u];
        if (PACKED) {
            const PackedTab T{words, 2 * SLOTS, cb, touched};
            c4_root<true>(g, vacc, u, ru.x, ru.y - ru.x, T, wid, NW, threadIdx.x, THREADS, seg, pv, flags);
        } else {
            const SplitTab T{reinterpret_cast<int *>(words), reinterpret_cast<int *>(words + SLOTS), SLOTS, touched};
            c4_root<true>(g, vacc, u, ru.x, ru.y - ru.x, T, wid, NW, threadIdx.x, THREADS, seg, pv, flags);
        }
    }
}

constexpr size_t cq_smem(int threads, int slots, int maxw) {
    // 2 x slots words, 2 x maxw 16-bit touched entries, segments, pv, flags
    return (size_t)2 * slots * 4 + (size_t)2 * maxw * 2 + (size_t)(threads / 32) * sizeof(SegTab) + 32 * 8 + 16;
}
constexpr size_t CM_SMEM = cq_smem(CM_THREADS, CM_SLOTS, CM_MAXW);
constexpr size_t CC_SMEM = cq_smem(CC_THREADS, CC_SLOTS, CC_MAXW);

// Both 128-thread queues in one launch: the packed one (W <= 6144 with
// enough count bits), then the split one (W <= 3072).
__global__ void __launch_bounds__(CM_THREADS) k_c4_mid(Graph g, VAcc *vacc, const int *lists, int *counters,
                                                       int cb) {
    pdl_begin();
    if (degree_overflow(counters)) return;
    c4_queue<CM_THREADS, CM_SLOTS, CM_MAXW, true>(g, vacc, lists + 5 * (size_t)g.n, counters[CNT_C4_MIDP],
                                                  counters + CNT_C4_MIDP_NEXT, cb);
    c4_queue<CM_THREADS, CM_SLOTS, CM_MAXW, false>(g, vacc, lists + 2 * (size_t)g.n, counters[CNT_C4_MID],
                                                   counters + CNT_C4_MID_NEXT, cb);
}

__global__ void __launch_bounds__(CC_THREADS) k_c4_cta(Graph g, VAcc *vacc, const int *lists, int *counters,
                                                       int cb) {
    pdl_begin();
    if (degree_overflow(counters)) return;
    c4_queue<CC_THREADS, CC_SLOTS, CC_MAXW, false>(g, vacc, lists + 3 * (size_t)g.n, counters[CNT_C4_CTA],
                                                   counters + CNT_C4_CTA_NEXT, cb);
}

// ------------------------------------------------------ key-tiled tier
//
// Roots with more wedges than the hash tiers take (W > teamw): one CTA per
// root, largest roots first. The keys w of a root u are the vertices below
// u; the CTA cuts them into tiles of TK consecutive ids and counts each
// tile's wedges in shared memory (16-bit counters while the root has fewer
// than 65535 in-neighbours, as no count exceeds that; 32-bit ones, half as
// many keys, above). A root's wedges through its in-neighbour v are the
// entries of row v below u, ascending, so the wedges that fall into a tile
// are a run of that row: every in-neighbour keeps a cursor (the start of its
// next run), the end of its wedge prefix and the key at the cursor. A tile
// first finds every in-neighbour's run (a galloping search from the cursor,
// one thread per in-neighbour) and its offset in the concatenation of the
// tile's runs (a prefix sum across the CTA); every warp then takes an equal
// slice of that concatenation, weighted so that each chunk of 32
// in-neighbours also counts for its overhead, and neither hub rows nor many
// short runs leave warps waiting.
// It counts the slice's wedges, credits C(c, 2) to every key w and to u
// from the counts, walks the slice again adding c - 1 per wedge to its
// middle vertex, moves the cursors past the runs, and clears. The next tile
// starts at the smallest key any cursor points at, so key ranges without
// wedges are skipped.
// The cursors of all these roots (their in-degrees sum to at most |E|) live
// in the region of the per-edge triangle counts, which nothing reads after
// the aggregate stage and which is sized 8 m bytes for them: 16 bytes per
// in-neighbour, |E| = m / 2 of them.
constexpr int CK_THREADS = 1024;
constexpr int CK_NW = CK_THREADS / 32;
constexpr size_t CK_OTHER = CK_NW * sizeof(SegTab) + CK_NW * 32 * 8 + 64 * 4;   // segment tables, sums, scalars
// Counter words (204 KB; tiles of 104448 keys with 16-bit counters). Larger
// tiles pay, as every tile costs passes over the in-neighbours: on R-MAT 22
// the tier took 598 ms with 48K words, 587 with 50K, 567 with 51K, and
// 571-572 with 51.5K and with all the 227 KB the rest leaves (52928).
constexpr int CK_WORDS = 51 * 1024;
constexpr int CK_NARROW_MAXD = 65534;               // in-degree up to which 16-bit counters cannot overflow
constexpr int CK_INF = 0x7fffffff;
// Weight of a chunk's overhead in elements when the walks are cut into warp
// slices: equal element counts left the warps of a tile with many short runs
// waiting at the tile barriers for the warp with the most chunks (R-MAT 22:
// 566 ms with equal elements; 430, 398, 372, 363, 367, 371, 392 ms with
// weights 32, 64, 128, 256, 384, 512, 1024).
constexpr int CK_ALPHA = 256;
constexpr size_t CK_SMEM = (size_t)CK_WORDS * 4 + CK_OTHER;
static_assert(CK_SMEM <= 227 * 1024, "k_c4_tiled shared memory");

// Root order of the key-tiled tier: the queued roots (list 4, their wedge
// counts in list 1) sorted by decreasing wedge count (64 buckets, two per
// octave) into list 0, and the prefix sums of their in-degrees (the offsets
// of their cursors) into list 2. One CTA.
__global__ void __launch_bounds__(1024) k_c4_tiled_plan(Graph g, int *lists, int *counters) {
    pdl_begin();
    __shared__ int hist[64], base[64];
    __shared__ int wsum[32];
    if (degree_overflow(counters)) return;
    const int nt = counters[CNT_C4_TEAM];
    if (nt == 0) return;
    const int *roots = lists + 4 * (size_t)g.n, *wts = lists + (size_t)g.n;
    int *sorted = lists, *offs = lists + 2 * (size_t)g.n;
    auto bucket = [](int w) {
        const int e = 31 - __clz(max(w, 1));
        const int half = e > 0 ? (w >> (e - 1)) & 1 : 0;
        return 63 - min(63, 2 * e + half);
    };
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) atomicAdd(&hist[bucket(wts[i])], 1);
    __syncthreads();
    if (threadIdx.x < 32) {   // exclusive scan of 64 buckets, two per lane
        const int a = hist[2 * threadIdx.x], b = hist[2 * threadIdx.x + 1];
        const int ex = warp_inclusive_scan(a + b) - (a + b);
        base[2 * threadIdx.x] = ex;
        base[2 * threadIdx.x + 1] = ex + a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) sorted[atomicAdd(&base[bucket(wts[i])], 1)] = roots[i];
    __syncthreads();
    int carry = 0;
    for (int j0 = 0; j0 < nt; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        int din = 0;
        if (j < nt) {
            const int4 r = g.rinfo[sorted[j]];
            din = r.y - r.x;
        }
        const int incl = warp_inclusive_scan(din);
        if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) wsum[threadIdx.x] = warp_inclusive_scan(wsum[threadIdx.x]);
        __syncthreads();
        const int before = (threadIdx.x >= 32 ? wsum[(threadIdx.x >> 5) - 1] : 0) + incl - din;
        if (j < nt) offs[j] = carry + before;
        carry += wsum[31];
        __syncthreads();
    }
}

// First position p in [cur, end) with a[p] >= key, given a[cur] < key
// (a ascending): doubling steps from cur, then a binary search.
__device__ __forceinline__ int gallop(const int *__restrict__ a, int cur, int end, int key) {
    int lo = cur, step = 1, hi = end;
    for (;;) {
        const int pr = lo + step;
        if (pr >= end) break;
        if (a[pr] >= key) {
            hi = pr;
            break;
        }
        lo = pr;
        step <<= 1;
    }
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid; else hi = mid;
    }
    return hi;
}

template <bool WIDE>
struct TileCounts {
    unsigned *c;
    __device__ __forceinline__ void add(int k) const {
        if (WIDE) atomicAdd(&c[k], 1u);
        else atomicAdd(&c[k >> 1], 1u << ((k & 1) << 4));
    }
    __device__ __forceinline__ int get(int k) const {
        return WIDE ? (int)c[k] : (int)((c[k >> 1] >> ((k & 1) << 4)) & 0xffffu);
    }
    static constexpr int keys_per_word = WIDE ? 1 : 2;
};

// One root of the key-tiled tier, the whole CTA. st: one int4 per
// in-neighbour {cursor, end of its wedge prefix, offset of its run in the
// tile's concatenation of runs, key at the cursor}. The offsets are scanned
// per warp over a contiguous range of R in-neighbours (R a multiple of 32,
// so a chunk never straddles two ranges); woff[r] turns range r's offsets
// into offsets in the whole tile.
template <bool WIDE>
__device__ __forceinline__ void c4_tiled_root(const Graph &g, VAcc *vacc, int u, int4 *st, unsigned *cnt,
                                              SegTab *segs, long long *pvs, int *ssm) {
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    const int4 ru = g.rinfo[u];
    const int b = ru.x, din = ru.y - ru.x;
    const int nch = (din + 31) >> 5;
    constexpr int TK = CK_WORDS * TileCounts<WIDE>::keys_per_word;
    const TileCounts<WIDE> T{cnt};
    SegTab &seg = segs[wid];
    long long *pv = pvs + wid * 32;
    int *woff = ssm, *s_next = ssm + 32, *s_tot = ssm + 33;
    const int RC = (din + 32 * CK_NW - 1) / (32 * CK_NW), R = RC * 32;   // chunks, in-neighbours per warp range
    auto offset = [&](int p) { return st[p].z + woff[p / R]; };   // p's run offset in the tile
    // cursors: each in-neighbour v's wedge prefix [row start, position of u in N+(v))
    int mn = CK_INF;
    for (int p = threadIdx.x; p < din; p += CK_THREADS) {
        const int v = g.ncol[b + p];
        const int4 rv = g.rinfo[v];
        const int e = lower_bound(g.ncol, rv.y, rv.z, u);
        const int nx = rv.x < e ? g.ncol[rv.x] : CK_INF;
        st[p] = make_int4(rv.x, e, 0, nx);
        mn = min(mn, nx);
    }
    pv[lane] = 0;
    mn = -warp_max(-mn);
    if (threadIdx.x == 0) *s_next = CK_INF;
    __syncthreads();
    if (lane == 0) atomicMin(s_next, mn);
    __syncthreads();
    int lo = *s_next;
    long long su = 0;
    // The wedges of elements [e0, e1) of the tile's concatenation of runs,
    // chunk by chunk of 32 in-neighbours: f(act, q, w) per wedge, done(v)
    // after each chunk.
    // Slices by weight: each chunk of 32 in-neighbours counts CK_ALPHA
    // elements of overhead ahead of its elements (its cursor loads, table
    // and window setup), so that a slice across many short runs gets fewer
    // elements. weighted() gives the chunk holding weighted position wp and
    // the element there.
    auto weighted = [&](long long wp, int total, long long &e) {
        int c = 0, top = nch;
        while (top - c > 1) {
            const int mid = (c + top) >> 1;
            if (offset(mid * 32) + (long long)CK_ALPHA * mid <= wp) c = mid; else top = mid;
        }
        const long long zc = offset(c * 32);
        const long long zn = c + 1 < nch ? offset((c + 1) * 32) : total;
        const long long x = wp - zc - (long long)CK_ALPHA * c - CK_ALPHA;
        e = zc + (x > 0 ? x : 0);
        if (e > zn) e = zn;
        return c;
    };
    auto visit = [&](long long e0, long long e1, int total, int c0, auto f, auto done) {
        if (e0 >= e1) return;
        int c = c0;
        int r = c / RC, left = RC - (c - r * RC);   // warp range of chunk c, chunks left in it
        for (; c < nch; ++c) {
            const int p = c * 32 + lane;
            int v = -1, cur = 0, end = 0, z = total;
            if (p < din) {
                const int4 s4 = st[p];
                cur = s4.x, end = s4.y, z = s4.z + woff[r];
                v = g.ncol[b + p];
            }
            const int cbase = __shfl_sync(FULL, z, 0);
            if (cbase >= e1) break;
            int znext = __shfl_down_sync(FULL, z, 1);
            if (lane == 31) znext = p + 1 < din ? st[p + 1].z + woff[left == 1 ? r + 1 : r] : total;
            if (--left == 0) {
                ++r;
                left = RC;
            }
            // the run, never past the in-neighbour's wedge prefix
            const int len = p < din ? min(max(znext - z, 0), end - cur) : 0;
            int pre;
            const int tot = seg_build(seg, cur, len, pre);
            const int from = (int)max(e0 - cbase, 0ll), to = (int)min(e1 - cbase, (long long)tot);
            if (from < to)
                seg_visit<4, true>(g.ncol, seg, pre, len, to, from, 32, [&](bool ok, int q, int, int w) { f(ok, q, w); });
            __syncwarp();
            done(v);
            __syncwarp();
        }
    };
    while (lo < u) {
        const int hi = min(lo + TK, u);
        const int nk = hi - lo;
        // A. every in-neighbour's run inside [lo, hi) (a galloping search from
        // its cursor) and the run's offset in the tile's concatenation: each
        // warp scans its range with a running carry, then one scan of the
        // warps' totals
        {
            int carry = 0;
            const int r0 = wid * R, r1 = min(r0 + R, din);
            for (int p0 = r0; p0 < r1; p0 += 32) {
                const int p = p0 + lane;
                int len = 0;
                if (p < r1) {
                    const int4 s4 = st[p];
                    if (s4.w < hi) len = gallop(g.ncol, s4.x, s4.y, hi) - s4.x;
                }
                const int incl = warp_inclusive_scan(len);
                if (p < r1) st[p].z = carry + incl - len;
                carry += __shfl_sync(FULL, incl, 31);
            }
            if (lane == 0) woff[wid] = carry;
            __syncthreads();
            if (wid == 0) {   // the warps' totals, CK_NW of them
                const int x = lane < CK_NW ? woff[lane] : 0;
                const int xi = warp_inclusive_scan(x);
                if (lane < CK_NW) woff[lane] = xi - x;
                if (lane == 31) *s_tot = xi;
            }
            __syncthreads();
        }
        const int total = *s_tot;
        // every warp takes an equal slice of the tile's weighted wedges (the
        // same slice for both walks)
        const long long wt = (long long)total + (long long)CK_ALPHA * nch;
        long long e0, e1;
        const int c0 = weighted(wt * wid / CK_NW, total, e0);
        weighted(wt * (wid + 1) / CK_NW, total, e1);
        if (wid == CK_NW - 1) e1 = total;
        // 1. count the tile's wedges
        visit(e0, e1, total, c0, [&](bool ok, int, int w) {
            if (ok && (unsigned)(w - lo) < (unsigned)nk) T.add(w - lo);   // always, for a simple graph
        }, [](int) {});
        __syncthreads();
        // 2. C(c, 2) to every key with c >= 2 and to u (the counts are only read from here on)
        const int nw4 = (nk + 4 * T.keys_per_word - 1) / (4 * T.keys_per_word);
        for (int i = threadIdx.x; i < nw4; i += CK_THREADS) {
            const uint4 q = reinterpret_cast<const uint4 *>(cnt)[i];
            if (!(q.x | q.y | q.z | q.w)) continue;
            const unsigned qw[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int h = 0; h < T.keys_per_word; ++h) {
                    const int c = WIDE ? (int)qw[j] : (int)((qw[j] >> (16 * h)) & 0xffffu);
                    if (c >= 2) {
                        const int k = (4 * i + j) * T.keys_per_word + h;
                        su += c2(c);
                        add64(&vacc[lo + k].C4, c2(c));
                    }
                }
            }
        }
        // 3. middle vertices: c - 1 per wedge, summed per in-neighbour
        visit(e0, e1, total, c0, [&](bool ok, int q, int w) {
            const bool in = ok && (unsigned)(w - lo) < (unsigned)nk;
            add_middle(pv, q, in ? T.get(w - lo) : 0);
        }, [&](int v) {
            const long long x = pv[lane];
            if (x) add64(&vacc[v].C4, x);
            pv[lane] = 0;
        });
        if (threadIdx.x == 0) *s_next = CK_INF;
        __syncthreads();
        // 4. cursors past the runs; the smallest next key starts the next
        // tile; clear the tile
        int tnext = CK_INF;
        for (int p = wid * R + lane; p < min((wid + 1) * R, din); p += 32) {   // the warp's own range
            const int4 s4 = st[p];
            const int z = s4.z + woff[wid];
            const int len = (p + 1 < din ? st[p + 1].z + woff[p + 1 == (wid + 1) * R ? wid + 1 : wid] : total) - z;
            int nx = s4.w;
            if (len > 0) {
                const int cur = s4.x + min(len, s4.y - s4.x);   // never past the wedge prefix
                nx = cur < s4.y ? g.ncol[cur] : CK_INF;
                st[p].x = cur;
                st[p].w = nx;
            }
            tnext = min(tnext, nx);
        }
        tnext = -warp_max(-tnext);
        if (lane == 0 && tnext < CK_INF) atomicMin(s_next, tnext);
        for (int i = threadIdx.x; i < nw4; i += CK_THREADS) reinterpret_cast<uint4 *>(cnt)[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        lo = *s_next;
        __syncthreads();
    }
    su = warp_sum(su);
    if (lane == 0 && su) add64(&vacc[u].C4, su);
    __syncthreads();
}

// cursors: room for `cap` entries; a list of roots whose in-degrees sum to
// more (only for a CSR that is not symmetric) stops with ENOTSIMPLE.
__global__ void __launch_bounds__(CK_THREADS) k_c4_tiled(Graph g, VAcc *vacc, const int *lists, int *counters,
                                                         int4 *cursors, long long cap, int *status) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char dsm[];
    unsigned *cnt = reinterpret_cast<unsigned *>(dsm);
    SegTab *segs = reinterpret_cast<SegTab *>(cnt + CK_WORDS);
    long long *pvs = reinterpret_cast<long long *>(segs + CK_NW);
    int *ssm = reinterpret_cast<int *>(pvs + CK_NW * 32);   // scan partials, next key, run total
    int *s_job = ssm + 40;
    if (degree_overflow(counters)) return;
    const int nt = counters[CNT_C4_TEAM];
    if (nt == 0) return;
    const int *sorted = lists, *offs = lists + 2 * (size_t)g.n;
    for (int i = threadIdx.x; i < CK_WORDS / 4; i += CK_THREADS)
        reinterpret_cast<uint4 *>(cnt)[i] = make_uint4(0, 0, 0, 0);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) *s_job = atomicAdd(&counters[CNT_C4_TILED_NEXT], 1);
        __syncthreads();
        const int j = *s_job;
        if (j >= nt) break;
        const int u = sorted[j];
        const int4 ru = g.rinfo[u];
        if ((long long)offs[j] + (ru.y - ru.x) > cap || offs[j] < 0) {
            if (threadIdx.x == 0) set_status(status, ST_ENOTSIMPLE);
            continue;
        }
        int4 *st = cursors + offs[j];
        if (ru.y - ru.x <= CK_NARROW_MAXD) c4_tiled_root<false>(g, vacc, u, st, cnt, segs, pvs, ssm);
        else c4_tiled_root<true>(g, vacc, u, st, cnt, segs, pvs, ssm);
    }
}

// Count bits of a packed table for ids below n: the key takes bits(n - 1).
static int packed_count_bits(int n) {
    unsigned top = n > 1 ? (unsigned)(n - 1) : 1u;
    int kb = 0;
    while (top) { ++kb; top >>= 1; }
    return 32 - kb;
}

void launch_cycle4(Work &w, cudaStream_t st) {
    // the wedge segments take the region of the triangle counts, dead after the aggregate stage
    int2 *wl = reinterpret_cast<int2 *>(w.tcnt);
    Graph g{w.n, w.m, w.rinfo, w.ncol, wl};
    if ((long long)w.m < 16ll * w.n) launch_pdl(k_c4_wedge_len<8>, w.num_sms * 8, 256, 0, st, g, wl, w.counters);
    else launch_pdl(k_c4_wedge_len<16>, w.num_sms * 8, 256, 0, st, g, wl, w.counters);
    after_launch(st, K_C4_WEDGE_LEN);
    int maxw = w.tune[TUNE_C4_WARP_MAXW] < CW_MAXW ? w.tune[TUNE_C4_WARP_MAXW] : CW_MAXW;
    // A graph with fewer vertices than the warp tier has resident warps is
    // bound by its slowest root's walk, one warp each: roots above
    // CW_SMALL_MAXW wedges go to the 4-warp tier there (G(2000, 0.01):
    // 104 -> 94 us per call).
    if (w.n <= w.num_sms * 32 && maxw > CW_SMALL_MAXW) maxw = CW_SMALL_MAXW;
    const int cb = packed_count_bits(w.n);
    // a packed word holds counts up to 2^cb - 2; with many vertices (large
    // graphs, batches) that is below what the warp tier takes, and the warp
    // tier counts in split tables instead
    const bool packed = (1ll << cb) - 2 >= maxw;
    const int teamw = w.tune[TUNE_C4_TEAM_MINW];
    static const int occ_w = resident_ctas((const void *)k_c4_warp, CW_WARPS * 32, 0);
    static const int occ_ws = resident_ctas((const void *)k_c4_warp_split, CW_WARPS * 32, 0);
    static const int occ_b = resident_ctas((const void *)k_c4_warp_big, CW_WARPS * 32, 0);
    static const int occ_bs = resident_ctas((const void *)k_c4_warp_big_split, CW_WARPS * 32, 0);
    if (packed)
        launch_pdl(k_c4_warp, w.num_sms * min(w.tune[TUNE_GRID_C4], occ_w), CW_WARPS * 32, 0, st, g, w.vacc, w.lists, w.counters, maxw,
                                                                             cb, teamw);
    else
        launch_pdl(k_c4_warp_split, w.num_sms * min(w.tune[TUNE_GRID_C4], occ_ws), CW_WARPS * 32, 0, st, g, w.vacc, w.lists, w.counters,
                                                                                   maxw, cb, teamw);
    after_launch(st, K_C4_WARP);
    // roots k_c4_warp queued for the 8 KB tables: one resident wave
    if (packed)
        launch_pdl(k_c4_warp_big, w.num_sms * occ_b, CW_WARPS * 32, 0, st, g, w.vacc, w.lists, w.counters, maxw, cb, teamw);
    else
        launch_pdl(k_c4_warp_big_split, w.num_sms * occ_bs, CW_WARPS * 32, 0, st, g, w.vacc, w.lists, w.counters, maxw, cb,
                                                                     teamw);
    after_launch(st, K_C4_WARP_BIG);
    static const int occ_m = resident_ctas((const void *)k_c4_mid, CM_THREADS, CM_SMEM);
    static const int occ_c = resident_ctas((const void *)k_c4_cta, CC_THREADS, CC_SMEM);
    launch_pdl(k_c4_mid, w.num_sms * occ_m, CM_THREADS, CM_SMEM, st, g, w.vacc, w.lists, w.counters, cb);
    after_launch(st, K_C4_MID);
    launch_pdl(k_c4_cta, w.num_sms * occ_c, CC_THREADS, CC_SMEM, st, g, w.vacc, w.lists, w.counters, cb);
    after_launch(st, K_C4_CTA);
    launch_pdl(k_c4_tiled_plan, 1, 1024, 0, st, g, w.lists, w.counters);
    after_launch(st, K_C4_PLAN);
    static const int occ_t = resident_ctas((const void *)k_c4_tiled, CK_THREADS, CK_SMEM);
    launch_pdl(k_c4_tiled, w.num_sms * occ_t, CK_THREADS, CK_SMEM, st, g, w.vacc, w.lists, w.counters,
                                                      reinterpret_cast<int4 *>(w.tcnt), (long long)w.m / 2,
                                                      w.status);
    after_launch(st, K_C4_TILED);
}

void configure_cycle4() {
    // the warp tiers need nearly all of an SM's shared memory for full residency
    cudaFuncSetAttribute(k_c4_warp, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_warp_split, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_warp_big, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_warp_big_split, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CM_SMEM);
    cudaFuncSetAttribute(k_c4_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC_SMEM);
    cudaFuncSetAttribute(k_c4_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CK_SMEM);
}

}  // namespace niorca
