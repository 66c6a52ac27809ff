// common.cuh -- device helpers shared by the NI-ORCA kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace niorca {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NCLASS = 128;  // degree classes used for the relabel order

// Device status bits (one per niorca_status code, bit k = code k).
enum : int {
    ST_EINVAL = 1 << 1,
    ST_ENOTSIMPLE = 1 << 2,
    ST_EOVERFLOW = 1 << 3,
    ST_ETIMEOUT = 1 << 6,
};

// Largest degree for which every intermediate of the orbit solve stays
// below 2^62 in int64 (each term is at most d_max^3 plus lower terms).
constexpr int MAX_DEGREE = 1 << 20;

// Degree class: exact for d < 8, then four classes per octave (the top two
// bits below the leading one). Classes are monotone in d, 0 <= class < 120.
__host__ __device__ __forceinline__ int deg_class(int d) {
    if (d < 8) return d < 0 ? 0 : d;
#ifdef __CUDA_ARCH__
    int e = 31 - __clz(d);
#else
    int e = 31 - __builtin_clz((unsigned)d);
#endif
    return 8 + (e - 3) * 4 + ((d >> (e - 2)) & 3);
}

// Per-vertex accumulators, indexed by the relabelled (degree-ordered) id.
// S1 and A1 come first: the orbit solve gathers them over neighbours.
struct __align__(16) VAcc {
    long long S1;   // sum of neighbour degrees
    long long A1;   // sum over incident edges of t_xy (= 2 * triangles at x)
    long long P6;   // sum over neighbours of C(d_y - 1, 2)
    long long A2;   // sum of t_xy^2
    long long A3;   // sum of t_xy * d_y
    long long D12;  // sum over triangles {x,y,z} of (t_yz - 1)   (f_12^14)
    long long K4;   // 4-cliques containing x                      (psi_14)
    long long C4;   // 4-cycles through x                          (psi_8)
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULL, v, o);
        if (lane_id() >= o) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

__device__ __forceinline__ void add64(long long *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

__device__ __forceinline__ void set_status(int *status, int bits) { atomicOr(status, bits); }

// Multiplicative hash of a vertex id into a power-of-two table (the sets of
// N+(u) in the triangle and aggregate stages, probed linearly: most probes
// there are misses that end at the first slot).
__device__ __forceinline__ unsigned hash_slot(int key, unsigned mask) {
    unsigned h = static_cast<unsigned>(key) * 0x9E3779B1u;
    return (h ^ (h >> 16)) & mask;
}

// Open-addressing set of vertex ids with a value (an index) per key, in
// buckets of 4 slots: a key hashes to a bucket and takes its first free
// slot, else the next bucket's. mask + 1 = slots, a power of two >= 4, at
// least twice the keys inserted, so probes always end; keys (16-byte
// aligned) are -1 when empty. Inserters try a bucket's slots in order, so
// a bucket fills from its first slot and one whose last slot is empty ends
// a search: at the loads used here (<= 1/2, mostly <= 1/4) a lookup is
// nearly always one 16-byte load with no probe loop.
__device__ __forceinline__ void hset_insert(int *keys, int *vals, unsigned mask, int key, int val) {
    const unsigned bmask = mask >> 2;
    unsigned b = hash_slot(key, bmask);
    for (unsigned probe = 0; probe <= bmask; ++probe) {
        for (unsigned j = 0; j < 4; ++j) {
            const int prev = atomicCAS(&keys[4 * b + j], -1, key);
            if (prev == -1 || prev == key) {
                vals[4 * b + j] = val;
                return;
            }
        }
        b = (b + 1) & bmask;
    }
}

__device__ __forceinline__ int hset_find(const int *keys, const int *vals, unsigned mask, int key) {
    const unsigned bmask = mask >> 2;
    unsigned b = hash_slot(key, bmask);
    for (unsigned probe = 0; probe <= bmask; ++probe) {
        const int4 k4 = reinterpret_cast<const int4 *>(keys)[b];
        const int j = k4.x == key ? 0 : k4.y == key ? 1 : k4.z == key ? 2 : k4.w == key ? 3 : -1;
        if (j >= 0) return vals[4 * b + j];
        if (k4.w == -1) return -1;
        b = (b + 1) & bmask;
    }
    return -1;
}

// Adds each run's sum of v to *p, once per run, where a run is a maximal
// group of adjacent lanes with the same key (the segments of a
// concatenation are such runs): the run's last lane adds the difference of
// the warp's inclusive scan at itself and before the run's first lane.
// Every lane calls it, each with its own key's p; v >= 0 and the sum over
// 32 lanes fits 32 bits. Grouping lanes with a warp match instead measured
// far slower on this GPU, and one atomic per lane serialises on a single
// 64-bit word when a whole window comes from one long row.
__device__ __forceinline__ void run_add(long long *p, int key, unsigned v) {
    const int lane = lane_id();
    const int kp = __shfl_up_sync(FULL, key, 1);
    const int kn = __shfl_down_sync(FULL, key, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0 || kp != key);
    const int rs = 31 - __clz(heads & ((2u << lane) - 1u));   // first lane of this lane's run
    const unsigned incl = warp_inclusive_scan(v);
    const unsigned before = __shfl_sync(FULL, incl - v, rs);
    if ((lane == 31 || kn != key) && incl != before)
        atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(incl - before));
}

// Per-warp table of the segments of one chunk (one segment per lane, e.g. the
// out-list of one neighbour), compacted to the non-empty ones in lane order:
// st = start position in the column array, pre = offset in the concatenation,
// idx = the lane that owns the segment.
struct SegTab {
    int st[32];
    int pre[32];
    int idx[32];
};

// Fills the table from each lane's segment (st, len); returns the length of
// the concatenation and the lane's own offset in `mypre`.
__device__ __forceinline__ int seg_build(SegTab &T, int st, int len, int &mypre) {
    const int incl = warp_inclusive_scan(len);
    mypre = incl - len;
    const unsigned ne = __ballot_sync(FULL, len > 0);
    if (len > 0) {
        const int r = __popc(ne & lanemask_lt());
        T.st[r] = st;
        T.pre[r] = mypre;
        T.idx[r] = lane_id();
    }
    __syncwarp();
    return __shfl_sync(FULL, incl, 31);
}

// Visits the concatenation in windows of 32 elements starting at wbase,
// wbase + stride, ... (wbase and stride warp-uniform multiples of 32), U
// windows per round with their loads issued first. The segment of element
// ws + lane is found without a search: one reduction marks where non-empty
// segments start inside the window, one ballot counts those that start
// before it. f(valid, q, pos, col[pos]) runs on every lane (q = owning lane).
// With COVER, a window that lies inside one segment (one ballot finds it)
// skips that lookup: its elements are contiguous in the segment's row. This
// pays where segments are long (hub rows) and costs a ballot where not.
template <int U, bool COVER = false, class F>
__device__ __forceinline__ void seg_visit(const int *__restrict__ col, const SegTab &T, int mypre, int mylen,
                                          int total, int wbase, int stride, F f) {
    const int lane = lane_id();
    const unsigned le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const unsigned ne = COVER ? __ballot_sync(FULL, mylen > 0) : 0u;   // lanes with a segment
    for (int w0 = wbase; w0 < total; w0 += U * stride) {
        int q[U], pos[U], val[U];
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const int ws = w0 + r * stride;
            if (COVER) {
                // (and ends within the walk: `total` may cut a segment)
                const unsigned cov =
                    __ballot_sync(FULL, ws + 32 <= total && mylen > 0 && mypre <= ws && mypre + mylen >= ws + 32);
                if (cov) {   // the segment of lane `src` holds the whole window
                    const int src = __ffs(cov) - 1;
                    const int rk = __popc(ne & ((1u << src) - 1u));
                    q[r] = src;
                    pos[r] = T.st[rk] - T.pre[rk] + ws + lane;
                    val[r] = __ldg(col + pos[r]);
                    continue;
                }
            }
            const bool starts = mylen > 0 && mypre >= ws && mypre < ws + 32;
            const unsigned sb = __reduce_or_sync(FULL, starts ? (1u << (mypre - ws)) : 0u);
            const int before = __popc(__ballot_sync(FULL, mylen > 0 && mypre < ws));
            const int k = ws + lane;
            q[r] = 0;
            pos[r] = -1;
            val[r] = 0;
            if (k < total) {
                const int rk = before + __popc(sb & le) - 1;
                q[r] = T.idx[rk];
                pos[r] = T.st[rk] + (k - T.pre[rk]);
                val[r] = __ldg(col + pos[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < U; ++r) f(pos[r] >= 0, q[r], pos[r], val[r]);
    }
}

// seg_visit for consecutive windows (stride 32) from wbase: a round of U
// windows takes its segment starts from one lane value (the start relative
// to the round), and the number of segments that start before a window is
// carried from the window before instead of counted by a ballot.
template <int U, class F>
__device__ __forceinline__ void seg_visit32(const int *__restrict__ col, const SegTab &T, int mypre, int mylen,
                                            int total, int wbase, F f) {
    const int lane = lane_id();
    const unsigned le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    int before = __popc(__ballot_sync(FULL, mylen > 0 && mypre < wbase));   // segments before the window
    for (int w0 = wbase; w0 < total; w0 += U * 32) {
        const int rel = mylen > 0 ? mypre - w0 : -1;   // this lane's segment start within the round
        const bool in_round = (unsigned)rel < (unsigned)(U * 32);
        int q[U], pos[U], val[U];
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const unsigned sb = __reduce_or_sync(FULL, in_round && (rel >> 5) == r ? 1u << (rel & 31) : 0u);
            const int k = w0 + 32 * r + lane;
            q[r] = 0;
            pos[r] = -1;
            val[r] = 0;
            if (k < total) {
                const int rk = before + __popc(sb & le) - 1;
                q[r] = T.idx[rk];
                pos[r] = T.st[rk] + (k - T.pre[rk]);
                val[r] = __ldg(col + pos[r]);
            }
            before += __popc(sb);
        }
#pragma unroll
        for (int r = 0; r < U; ++r) f(pos[r] >= 0, q[r], pos[r], val[r]);
    }
}

// First position p in [lo, hi) with a[p] >= key (a sorted ascending).
__device__ __forceinline__ int lower_bound(const int *a, int lo, int hi, int key) {
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Position of key in sorted a[lo, hi), or -1.
__device__ __forceinline__ int find_sorted(const int *a, int lo, int hi, int key) {
    int p = lower_bound(a, lo, hi, key);
    return (p < hi && a[p] == key) ? p : -1;
}

__host__ __device__ __forceinline__ unsigned next_pow2(unsigned v) {
    v--;
    v |= v >> 1; v |= v >> 2; v |= v >> 4; v |= v >> 8; v |= v >> 16;
    return v + 1;
}

// Work-memory views of one counting call (all device pointers).
// rinfo[u] = {row start, split, row end, 0} of the relabelled row of u:
// N-(u) = ncol[x, y), N+(u) = ncol[y, z), one 16-byte load per row.
struct Graph {
    int n;              // vertices
    int m;              // CSR entries (2|E|)
    const int4 *rinfo;  // row bounds of every relabelled vertex
    const int *ncol;    // relabelled neighbours, rows ascending
    const int2 *wl = nullptr;  // 4-cycle stage: at the position of in-neighbour v in row u (rows with at most
                               // WL_MAXD in-neighbours), {start of row v, number of entries of row v below u}
};
constexpr int WL_MAXD = 1024;

}  // namespace niorca
