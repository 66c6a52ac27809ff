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
// (k_c4_midp / k_c4_mid), a 512-thread CTA (k_c4_cta), or a cluster of
// CTAs sharing a dense count row in global memory (k_c4_team). The other tables are open-addressing hash tables in
// shared memory, either split (key and count arrays) or packed (key << cb |
// count in one 32-bit word, cb = 32 - bits(n - 1) count bits, usable while
// W < 2^cb - 1), which holds twice the keys in the same space. Each table
// is emptied once per CTA; afterwards a warp sweeps the region its root
// used, and a CTA empties the slots it filled (kept in a 16-bit `touched`
// list).
#include <cooperative_groups.h>

#include "kernels.h"

namespace niorca {

constexpr int CW_WARPS = 4;
constexpr int CW_WORDS = 1536;      // table words per warp of k_c4_warp: 6 KB, 8 CTAs of 4 warps per SM
constexpr int CWB_WORDS = 2048;     // k_c4_warp_big: 8 KB, 6 CTAs per SM
constexpr int CW_MAXW = 1536;       // largest W of a root in the warp tiers
constexpr int CW_DUPS = 32;         // repeated keys a warp credits without a second walk
constexpr int CW_BIG_LIST = 0;      // list slot of k_c4_warp_big's roots: the triangle stage's heavy list,
                                    // which nothing reads after that stage
constexpr int CM_THREADS = 128;
constexpr int CM_SLOTS = 4096;      // split; 8192 when packed
constexpr int CM_MAXW = 3072;      // split; 6144 when packed
constexpr int CC_THREADS = 512;
constexpr int CC_SLOTS = 16384;     // split
constexpr int CC_MAXW = 12288;
constexpr int CT_THREADS = 1024;   // team tier: CTAs of a cluster share one dense row
constexpr int CT_CLUSTER = 8;
constexpr int CT_MAXCH = (1 << 20) / 32;   // chunks of 32 in-neighbours (degree <= 2^20)
constexpr size_t CT_SMEM = (size_t)(CT_MAXCH + 1) * 4;
constexpr unsigned EMPTY = 0xffffffffu;

__device__ __forceinline__ long long c2(long long c) { return c * (c - 1) / 2; }

// Adds c - 1 to pv[q] for the lanes with c > 1: one warp-aggregated atomic
// per in-neighbour when many lanes take part (long rows of hub roots), plain
// shared atomics when few do.
__device__ __forceinline__ void add_middle(long long *pv, int q, int c) {
    const unsigned m = __ballot_sync(FULL, c > 1);
    if (!m) return;
    if (__popc(m) > 8) warp_add_ll(c > 1, &pv[q], q, c - 1);
    else if (c > 1) atomicAdd(reinterpret_cast<unsigned long long *>(&pv[q]), (unsigned long long)(c - 1));
}

// Wedges u - v - w through the in-neighbour v of root u: the entries of row
// v below u, i.e. the position of u in row v (u is in N+(v)), found by a
// search of N+(v) whose last steps touch the lines the walk reads next.
__device__ __forceinline__ int wedge_len(const Graph &g, int u, const int4 &rv) {
    return lower_bound(g.ncol, rv.y, rv.z, u) - rv.x;
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
        const int4 rv = g.rinfo[v];
        st = rv.x;
        len = wedge_len(g, u, rv);
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
        seg_visit<4>(g.ncol, T, pre, len, total, 0, 32, [&](bool ok, int q, int, int w) { f(ok, q, w); });
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
// keeps no list: its table is sized to the root (at least twice W slots),
// and it sweeps that region.
// pv holds the per-middle-vertex sums of one chunk (per warp, or shared by
// the CTA).
template <bool CTA, class Tab>
__device__ __forceinline__ void c4_root(const Graph &g, VAcc *vacc, int u, int b, int din,
                                        const Tab &T, int wid, int nw, int tid, int nthreads, SegTab &seg,
                                        long long *pv, int *flags, const RootChunks &rc = RootChunks{}) {
    const int lane = lane_id();
    auto sync = [] {
        if (CTA) __syncthreads(); else __syncwarp();
    };
    bool dup_l = false;   // warp group: this lane saw a repeated key
    auto insert = [&](bool act, int, int w) {
        const int slot = act ? T.add(w) : -2;
        if (!CTA) {
            dup_l |= slot == -1;
            return;
        }
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
    if (!CTA && __any_sync(FULL, dup_l)) {
        // A warp sweeps its table for the repeated keys (count >= 2), credits
        // them, and lists up to CW_DUPS of them in flags[]; the middle
        // vertices of key w are N-(u) ∩ N(w), found by searching row w for
        // each in-neighbour. More repeated keys: the middle walk below.
        long long su = 0;
        int nd = 0;
        for (int i0 = 0; i0 < nt; i0 += 32) {   // all lanes take part in every ballot
            const int i = i0 + lane;
            const int c = (i >= nt || T.empty(i)) ? 0 : T.cnt(i);
            const unsigned rep = __ballot_sync(FULL, c >= 2);
            if (c >= 2) {
                const int w = T.key(i);
                su += c2(c);
                add64(&vacc[w].C4, c2(c));
                const int k = nd + __popc(rep & lanemask_lt());
                if (k < CW_DUPS) {
                    flags[k] = w;
                    flags[CW_DUPS + k] = c;
                }
            }
            nd += __popc(rep);
        }
        su = warp_sum(su);
        if (lane == 0) add64(&vacc[u].C4, su);
        __syncwarp();
        if (nd <= CW_DUPS) {
            for (int k = 0; k < nd; ++k) {
                const int w = flags[k], c = flags[CW_DUPS + k];
                const int4 rw = g.rinfo[w];
                for (int ch = 0, p = lane; p < din; ++ch, p += 32) {
                    const int v = ch < rc.have ? (ch == 0 ? rc.v0 : rc.v1) : g.ncol[b + p];
                    if (find_sorted(g.ncol, rw.x, rw.z, v) >= 0) add64(&vacc[v].C4, c - 1);
                }
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

constexpr int CW_MIN_SLOTS = 64;

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
__device__ __forceinline__ void c4_warp_body(Graph g, VAcc *vacc, int *lists, int *counters, int maxw, int cb) {
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
    int v0 = (i < count && lane < ru.y - ru.x) ? g.ncol[ru.x + lane] : -1;
    int4 rv0 = v0 >= 0 ? g.rinfo[v0] : Z;
    for (; i < count; i += nw) {
        const int i2 = i + 2 * nw;
        const int u2 = i2 < count ? root(i2) : 0;
        const int4 ru2 = i2 < count ? g.rinfo[u2] : Z;
        const int v1 = (i + nw < count && lane < ru1.y - ru1.x) ? g.ncol[ru1.x + lane] : -1;
        int4 rv1 = Z;
        bool rv1_loaded = false;
        [&] {
            const int b = ru.x, din = ru.y - ru.x;
            if (din < 2) return;
            long long W = 0;   // exact wedge count W of root u
            RootChunks rc;
            if (din <= 64) {   // both chunks' segments stay in registers
                rc.v0 = v0;
                if (lane < din) {
                    rc.st0 = rv0.x;
                    rc.len0 = wedge_len(g, u, rv0);
                }
                if (din <= 32) {   // one chunk: its segment table gives W
                    rc.have = 1;
                    rc.total0 = seg_build(S.seg, rc.st0, rc.len0, rc.pre0);
                    rc.built0 = true;
                    W = rc.total0;
                } else {
                    rc.have = 2;
                    if (32 + lane < din) {
                        rc.v1 = g.ncol[b + 32 + lane];
                        const int4 r1 = g.rinfo[rc.v1];
                        rc.st1 = r1.x;
                        rc.len1 = wedge_len(g, u, r1);
                    }
                    W = warp_sum(rc.len0 + rc.len1);
                }
            } else {
                for (int p = lane; p < din; p += 32) W += wedge_len(g, u, g.rinfo[g.ncol[b + p]]);
                W = warp_sum(W);
            }
            rv1 = v1 >= 0 ? g.rinfo[v1] : Z;   // next root's in-neighbours, during this walk
            rv1_loaded = true;
            if (W < 2) return;
            if (W > here_lim) {
                if (lane == 0) {
                    int which, list;   // queue counter and list slot (lists + list * n)
                    if (!BIG && W <= big_lim) { which = CNT_C4_WBIG; list = CW_BIG_LIST; }
                    else if (W > CC_MAXW) { which = CNT_C4_TEAM; list = 4; }
                    else if (W <= 2 * CM_MAXW && W <= pack_lim) { which = CNT_C4_MIDP; list = 5; }
                    else if (W <= CM_MAXW) { which = CNT_C4_MID; list = 2; }
                    else { which = CNT_C4_CTA; list = 3; }
                    lists[(size_t)list * g.n + atomicAdd(&counters[which], 1)] = u;
                }
                return;
            }
            // at least 2W slots (W <= half the table), else the whole table (W <= 3/4 of it)
            unsigned slots = next_pow2(2 * (unsigned)W);
            slots = slots < CW_MIN_SLOTS ? CW_MIN_SLOTS : (slots > (unsigned)TS ? (unsigned)TS : slots);
            if constexpr (SPLIT) {
                const SplitTab T{sk, sc, slots, nullptr};
                c4_root<false>(g, vacc, u, b, din, T, 0, 1, lane, 32, S.seg, S.pv, S.dups, rc);
            } else {
                const PackedTab T{S.t, slots, cb, nullptr};
                c4_root<false>(g, vacc, u, b, din, T, 0, 1, lane, 32, S.seg, S.pv, S.dups, rc);
            }
        }();
        if (!rv1_loaded) rv1 = v1 >= 0 ? g.rinfo[v1] : Z;
        u = un;
        un = u2;
        ru = ru1;
        ru1 = ru2;
        v0 = v1;
        rv0 = rv1;
    }
}

// 8 CTAs of 4 warps per SM: 6 KB tables and at most 64 registers a thread.
__global__ void __launch_bounds__(CW_WARPS * 32, 8) k_c4_warp(Graph g, VAcc *vacc, int *lists, int *counters,
                                                              int maxw, int cb) {
    c4_warp_body<false, false>(g, vacc, lists, counters, maxw, cb);
}

__global__ void __launch_bounds__(CW_WARPS * 32, 8) k_c4_warp_split(Graph g, VAcc *vacc, int *lists,
                                                                    int *counters, int maxw, int cb) {
    c4_warp_body<true, false>(g, vacc, lists, counters, maxw, cb);
}

__global__ void __launch_bounds__(CW_WARPS * 32) k_c4_warp_big(Graph g, VAcc *vacc, int *lists, int *counters,
                                                               int maxw, int cb) {
    c4_warp_body<false, true>(g, vacc, lists, counters, maxw, cb);
}

__global__ void __launch_bounds__(CW_WARPS * 32) k_c4_warp_big_split(Graph g, VAcc *vacc, int *lists,
                                                                     int *counters, int maxw, int cb) {
    c4_warp_body<true, true>(g, vacc, lists, counters, maxw, cb);
}

// Roots from a queue, one CTA each. The table (SLOTS split slots, or
// 2 x SLOTS packed ones) lives in dynamic shared memory and is emptied once
// per CTA.
template <int THREADS, int SLOTS, int MAXW, bool PACKED>
__device__ __forceinline__ void c4_queue(const Graph &g, VAcc *vacc, const int *list, int count,
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
    for (int h = blockIdx.x; h < count; h += gridDim.x) {
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

__global__ void __launch_bounds__(CM_THREADS) k_c4_mid(Graph g, VAcc *vacc, const int *lists,
                                                       const int *counters, int cb) {
    c4_queue<CM_THREADS, CM_SLOTS, CM_MAXW, false>(g, vacc, lists + 2 * (size_t)g.n, counters[CNT_C4_MID], cb);
}

__global__ void __launch_bounds__(CM_THREADS) k_c4_midp(Graph g, VAcc *vacc, const int *lists,
                                                        const int *counters, int cb) {
    c4_queue<CM_THREADS, CM_SLOTS, CM_MAXW, true>(g, vacc, lists + 5 * (size_t)g.n, counters[CNT_C4_MIDP], cb);
}

__global__ void __launch_bounds__(CC_THREADS) k_c4_cta(Graph g, VAcc *vacc, const int *lists,
                                                       const int *counters, int cb) {
    c4_queue<CC_THREADS, CC_SLOTS, CC_MAXW, false>(g, vacc, lists + 3 * (size_t)g.n, counters[CNT_C4_CTA], cb);
}

// Zero the dense rows of the team tier (only when that tier has work).
__global__ void k_c4_zero_dense(int *dense, long long words, const int *counters) {
    if (counters[CNT_C4_TEAM] == 0) return;
    int4 *d4 = reinterpret_cast<int4 *>(dense);
    const long long n4 = words / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        d4[i] = make_int4(0, 0, 0, 0);
    for (long long i = n4 * 4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < words;
         i += (long long)gridDim.x * blockDim.x)
        dense[i] = 0;
}

// Roots with W > CC_MAXW: one cluster of CT_CLUSTER CTAs per root, counting
// in a dense row of n ints in global memory that the cluster shares, so
// that only one row per cluster is live. The root's wedges, in the order
// of its in-neighbours, are cut into equal slices, one per warp of the
// cluster; every CTA keeps the prefix sums of the wedge counts of the
// root's 32-in-neighbour chunks (W < 2^31: a root's wedges are entries of
// rows of the CSR) to find where a slice starts.
// Pass 1 adds every wedge; pass 2 reads each count (per middle vertex) and
// marks the key with the sign bit, so that exactly one visitor credits
// C(c, 2) to w; pass 3 stores zeros back. Cluster barriers separate the
// passes.
__global__ void __cluster_dims__(CT_CLUSTER, 1, 1) __launch_bounds__(CT_THREADS)
    k_c4_team(Graph g, VAcc *vacc, const int *lists, const int *counters, int *dense, int teams) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    constexpr int NW = CT_THREADS / 32;
    constexpr int SLICES = NW * CT_CLUSTER;
    extern __shared__ __align__(16) unsigned char dsm[];
    int *P = reinterpret_cast<int *>(dsm);   // chunk prefix sums, CT_MAXCH + 1
    __shared__ SegTab segs[NW];
    __shared__ long long pvs[NW][32];
    __shared__ int wsum[NW];
    const int team = blockIdx.x / CT_CLUSTER;
    const int wid = threadIdx.x >> 5, lane = lane_id();
    const int slice = (int)cluster.block_rank() * NW + wid;
    int *row = dense + (size_t)team * g.n;
    SegTab &seg = segs[wid];
    long long *pv = pvs[wid];
    const int *glob_list = lists + 4 * (size_t)g.n;
    const int nh = counters[CNT_C4_TEAM];
    for (int h = team; h < nh; h += teams) {
        const int u = glob_list[h];
        const int4 ru = g.rinfo[u];
        const int b = ru.x, din = ru.y - ru.x;
        const int nch = (din + 31) >> 5;
        // wedges per chunk (P[c]), then an exclusive scan in place: each
        // thread owns a run of consecutive chunks, and only it touches them
        for (int c = wid; c < nch; c += NW) {
            const int p = c * 32 + lane;
            const int l = p < din ? wedge_len(g, u, g.rinfo[g.ncol[b + p]]) : 0;
            const int sum = warp_sum(l);
            if (lane == 0) P[c] = sum;
        }
        __syncthreads();
        {
            const int per = (nch + CT_THREADS - 1) / CT_THREADS;
            const int c0 = min(threadIdx.x * per, nch), c1 = min(c0 + per, nch);
            int run = 0;
            for (int c = c0; c < c1; ++c) run += P[c];
            const int incl = warp_inclusive_scan(run);
            if (lane == 31) wsum[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                const int x = wsum[lane];
                wsum[lane] = warp_inclusive_scan(x) - x;
            }
            __syncthreads();
            int acc = wsum[wid] + incl - run;
            for (int c = c0; c < c1; ++c) {
                const int t = P[c];
                P[c] = acc;
                acc += t;
            }
            if (c0 < c1 && c1 == nch) P[nch] = acc;   // W
        }
        __syncthreads();
        const int W = P[nch];
        const int lo = (int)((long long)W * slice / SLICES), hi = (int)((long long)W * (slice + 1) / SLICES);
        // chunks overlapping [lo, hi): f(act, q, w) per wedge, done(v) per chunk
        auto pass = [&](auto f, auto done) {
            if (lo >= hi) return;
            int c = 0, top = nch;   // last chunk with P[c] <= lo
            while (top - c > 1) {
                const int mid = (c + top) >> 1;
                if (P[mid] <= lo) c = mid; else top = mid;
            }
            for (; c < nch && P[c] < hi; ++c) {
                int v, len, pre;
                const int total = wedge_chunk(g, u, b, din, c * 32, seg, v, len, pre);
                const int from = max(lo - P[c], 0), to = min(hi - P[c], total);
                seg_visit<4>(g.ncol, seg, pre, len, to, from, 32, [&](bool ok, int q, int, int w) { f(ok, q, w); });
                __syncwarp();
                done(v);
                __syncwarp();
            }
        };
        // Roots with many wedges for their row (W > u / 16) read the counts
        // back in a coalesced sweep of row[0, u) for the C(c, 2) credits and
        // with plain loads for the middle sums, and clear the row with a
        // coalesced sweep; others mark first visitors and clear per wedge.
        const bool sweep = (long long)W * 16 > u;
        const int gt = (int)cluster.block_rank() * CT_THREADS + threadIdx.x;
        constexpr int GT = CT_CLUSTER * CT_THREADS;
        pass([&](bool act, int, int w) { if (act) atomicAdd(&row[w], 1); }, [](int) {});
        cluster.sync();
        long long su = 0;
        pv[lane] = 0;
        __syncwarp();
        auto flush = [&](int v) {
            const long long x = pv[lane];
            if (x) add64(&vacc[v].C4, x);
            pv[lane] = 0;
        };
        if (sweep) {
            for (int w = gt; w < u; w += GT) {
                const int c = row[w];
                if (c >= 2) {
                    su += c2(c);
                    add64(&vacc[w].C4, c2(c));
                }
            }
            pass([&](bool act, int q, int w) { add_middle(pv, q, act ? row[w] : 0); }, flush);
        } else pass(
            [&](bool act, int q, int w) {
                int c = 0;
                if (act) {
                    const int old = atomicOr(&row[w], (int)0x80000000);
                    c = old & 0x7fffffff;
                    if (old >= 0 && c >= 2) {   // first visitor of this key
                        su += c2(c);
                        add64(&vacc[w].C4, c2(c));
                    }
                }
                add_middle(pv, q, c);   // lanes of one v add once
            },
            flush);
        su = warp_sum(su);
        if (lane == 0 && su) add64(&vacc[u].C4, su);
        cluster.sync();
        if (sweep) {
            for (int w = gt; w < u; w += GT) row[w] = 0;
        } else {
            pass([&](bool act, int, int w) { if (act) row[w] = 0; }, [](int) {});
        }
        cluster.sync();
    }
}

// One dense row per cluster, as many clusters as the SMs hold, but no more
// rows than about 200 MB (1.5 times the L2) hold: the rows' atomics then
// mostly stay in L2. On R-MAT scale 22 (16.8 MB a row) 11 rows instead of
// 19 take 9% off this tier; 5 rows, all in L2, leave too few SMs working
// and take twice as long.
int c4_team_rows(int num_sms, long long n) {
    int t = num_sms / CT_CLUSTER;
    const long long fit = 200000000ll / (4 * (n > 0 ? n : 1));
    if (fit < t) t = (int)fit;
    return t < 1 ? 1 : t;
}

// Count bits of a packed table for ids below n: the key takes bits(n - 1).
static int packed_count_bits(int n) {
    unsigned top = n > 1 ? (unsigned)(n - 1) : 1u;
    int kb = 0;
    while (top) { ++kb; top >>= 1; }
    return 32 - kb;
}

void launch_cycle4(Work &w, cudaStream_t st) {
    Graph g{w.n, w.m, w.rinfo, w.ncol};
    const int maxw = w.tune[TUNE_C4_WARP_MAXW] < CW_MAXW ? w.tune[TUNE_C4_WARP_MAXW] : CW_MAXW;
    const int cb = packed_count_bits(w.n);
    // a packed word holds counts up to 2^cb - 2; with many vertices (large
    // graphs, batches) that is below what the warp tier takes, and the warp
    // tier counts in split tables instead
    const bool packed = (1ll << cb) - 2 >= maxw;
    if (packed)
        k_c4_warp<<<w.num_sms * w.tune[TUNE_GRID_C4], CW_WARPS * 32, 0, st>>>(g, w.vacc, w.lists, w.counters, maxw,
                                                                             cb);
    else
        k_c4_warp_split<<<w.num_sms * w.tune[TUNE_GRID_C4], CW_WARPS * 32, 0, st>>>(g, w.vacc, w.lists, w.counters,
                                                                                   maxw, cb);
    after_launch(st, K_C4_WARP);
    // roots k_c4_warp queued for the 8 KB tables: one resident wave
    if (packed)
        k_c4_warp_big<<<w.num_sms * 6, CW_WARPS * 32, 0, st>>>(g, w.vacc, w.lists, w.counters, maxw, cb);
    else
        k_c4_warp_big_split<<<w.num_sms * 6, CW_WARPS * 32, 0, st>>>(g, w.vacc, w.lists, w.counters, maxw, cb);
    after_launch(st, K_C4_WARP_BIG);
    k_c4_midp<<<w.num_sms * 4, CM_THREADS, CM_SMEM, st>>>(g, w.vacc, w.lists, w.counters, cb);
    after_launch(st, K_C4_MIDP);
    k_c4_mid<<<w.num_sms * 4, CM_THREADS, CM_SMEM, st>>>(g, w.vacc, w.lists, w.counters, cb);
    after_launch(st, K_C4_MID);
    k_c4_cta<<<w.num_sms, CC_THREADS, CC_SMEM, st>>>(g, w.vacc, w.lists, w.counters, cb);
    after_launch(st, K_C4_CTA);
    if (w.c4slots > 0) {
        const long long words = (long long)c4_dense_words(w.c4slots, w.n);
        k_c4_zero_dense<<<w.num_sms * 4, 256, 0, st>>>(w.c4dense, words, w.counters);
        after_launch(st, K_C4_ZERO);
        k_c4_team<<<w.c4slots * CT_CLUSTER, CT_THREADS, CT_SMEM, st>>>(g, w.vacc, w.lists, w.counters,
                                                                       w.c4dense, w.c4slots);
        after_launch(st, K_C4_TEAM);
    }
}

void configure_cycle4() {
    // the warp tiers need nearly all of an SM's shared memory for full residency
    cudaFuncSetAttribute(k_c4_warp, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_warp_split, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_warp_big, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_warp_big_split, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_c4_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CM_SMEM);
    cudaFuncSetAttribute(k_c4_midp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CM_SMEM);
    cudaFuncSetAttribute(k_c4_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC_SMEM);
    cudaFuncSetAttribute(k_c4_team, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT_SMEM);
}

}  // namespace niorca
