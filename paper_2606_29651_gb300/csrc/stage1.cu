// stage1.cu -- Stage I (per-edge triangle counts, Algorithm 1) fused with
// Stage II (K4 per vertex, Algorithm 2).
//
// In the relabelled graph every triangle u < v < w is found once, at its
// lowest vertex u, as w in N+(u) ∩ N+(v) (Algorithm 2 enumerates the same
// way with ids). For a root u the kernel loads N+(u) into a shared-memory
// hash table, streams N+(v) of every v in N+(u) across the lanes of a warp
// (the lists of several v are concatenated so that every lane is busy) and
// probes each element. A hit is a triangle (u, v, w): t(v,w) is added to
// global memory at the position of w in row v, and the hit sets bit i of row
// j of R, the adjacency bit-matrix of N+(u) oriented upwards (R[j] bit i <=>
// N+(u)[i] in N+(N+(u)[j]), v = N+(u)[j], w = N+(u)[i]).
// In the warp tier t(u,v) and t(u,w) are also counted in shared memory per
// hit, and a K4 u < v < w < x is a triangle (j, i) of R together with a
// common bit of R[j] and R[i] -- Algorithm 2's pairwise test over `neigh`
// done as word-wide bit operations. In the CTA tiers R is mirrored after the
// expansion (a ballot transpose per 32 x 32 block), t(u, N+(u)[y]) is the
// popcount of row y, and the K4s of u through y are the triangles of R at y:
// twice their number is the sum over the neighbours z of y in R of
// popc(R[y] & R[z]). A warp takes a row and its lanes one neighbour z each,
// with the same word loop on every lane, so the cost follows the edges of R
// and not the (much larger) number of K4s of dense hub neighbourhoods.
#include "kernels.h"

namespace niorca {

// ----------------------------------------------------------- warp tier

constexpr int TW_MAXD = 64;   // out-degree handled by one warp
constexpr int TS_MAXD = 256;  // out-degree handled by a 256-thread CTA (k_tri_cta)
constexpr int TW_WARPS = 8;

struct __align__(16) TriWarpSmem {
    int hk[4 * TW_MAXD];   // N+(u) hash at load <= 1/4 (most probes are misses)
    int hv[4 * TW_MAXD];
    int cnt[TW_MAXD];
    int kc[TW_MAXD];
    unsigned R[TW_MAXD][2];
    SegTab seg;
};

__global__ void __launch_bounds__(TW_WARPS * 32, 8) k_tri_warp(Graph g, int *tcnt, VAcc *vacc, int *heavy,
                                                            int *counters, int maxd) {
    pdl_begin();
    __shared__ TriWarpSmem sm_all[TW_WARPS];
    TriWarpSmem &S = sm_all[threadIdx.x >> 5];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (degree_overflow(counters)) return;
    for (int u = gw; u < g.n; u += nw) {
        const int4 ru = g.rinfo[u];
        const int s = ru.y, e = ru.z, dp = e - s;
        if (dp < 2) continue;
        if (dp > maxd) {
            if (lane == 0) {
                if (dp <= TS_MAXD) heavy[atomicAdd(&counters[CNT_TRI_HEAVY], 1)] = u;
                else heavy[g.n - 1 - atomicAdd(&counters[CNT_TRI_BIG], 1)] = u;
            }
            continue;
        }
        const unsigned mask = next_pow2(4 * dp) - 1;
        for (int i = lane; i <= (int)mask; i += 32) S.hk[i] = -1;
        for (int i = lane; i < TW_MAXD; i += 32) {
            S.cnt[i] = 0;
            S.kc[i] = 0;
            S.R[i][0] = 0;
            S.R[i][1] = 0;
        }
        __syncwarp();
        for (int i = lane; i < dp; i += 32) hset_insert(S.hk, S.hv, mask, g.ncol[s + i], i);
        const int umax = g.ncol[e - 1];
        __syncwarp();
        int found = 0;
        for (int jb = 0; jb < dp - 1; jb += 32) {   // the last out-neighbour has no row to walk
            const int j = jb + lane;
            int len = 0, vs = 0;
            if (j < dp - 1) {
                const int4 rv = g.rinfo[g.ncol[s + j]];
                vs = rv.y;
                len = rv.z - rv.y;
            }
            int mypre;
            const int total = seg_build(S.seg, vs, len, mypre);
            seg_visit32<2>(g.ncol, S.seg, mypre, len, total, 0, [&](bool valid, int q, int pos, int w) {
                const int i = (valid && w <= umax) ? hset_find(S.hk, S.hv, mask, w) : -1;
                const bool hit = i >= 0;
                if (!__any_sync(FULL, hit)) return;
                const int jj = jb + q;
                if (hit) {
                    atomicAdd(&S.cnt[jj], 1);
                    atomicOr(&S.R[0][0] + jj * 2 + (i >> 5), 1u << (i & 31));
                    atomicAdd(&S.cnt[i], 1);
                    atomicAdd(&tcnt[pos], 1);
                    found = 1;
                }
            });
            __syncwarp();
        }
        if (!__any_sync(FULL, found)) continue;
        for (int i = lane; i < dp; i += 32)
            if (S.cnt[i]) atomicAdd(&tcnt[s + i], S.cnt[i]);
        long long ku = 0;
        for (int j = lane; j < dp; j += 32) {
            const unsigned rj0 = S.R[j][0], rj1 = S.R[j][1];
            for (int wd = 0; wd < 2; ++wd) {
                unsigned bits = wd ? rj1 : rj0;
                while (bits) {
                    const int i = wd * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    unsigned x0 = rj0 & S.R[i][0], x1 = rj1 & S.R[i][1];
                    const int k = __popc(x0) + __popc(x1);
                    if (!k) continue;
                    ku += k;
                    atomicAdd(&S.kc[j], k);
                    atomicAdd(&S.kc[i], k);
                    while (x0) { atomicAdd(&S.kc[__ffs(x0) - 1], 1); x0 &= x0 - 1; }
                    while (x1) { atomicAdd(&S.kc[32 + __ffs(x1) - 1], 1); x1 &= x1 - 1; }
                }
            }
        }
        ku = warp_sum(ku);
        __syncwarp();
        if (lane == 0 && ku) add64(&vacc[u].K4, ku);
        for (int i = lane; i < dp; i += 32)
            if (S.kc[i]) add64(&vacc[g.ncol[s + i]].K4, S.kc[i]);
        __syncwarp();
    }
}

// ------------------------------------------------------------ CTA tiers

// Roots with out-degree above the warp tier get a CTA each, in two sizes:
// k_tri_cta (256 threads, dp <= TS_MAXD) needs about 18 KB of shared memory,
// so several CTAs share an SM; k_tri_big (1024 threads) takes the rest with
// the bit matrix R up to TB_BITMAT_MAXD (hash of N+(u) capped at 4096 slots),
// a 16384-slot hash up to TB_HASH_MAXD, and binary searches beyond.
// k_tri_warp queues the first kind from the front of the heavy list and the
// second from its back.
constexpr int TS_THREADS = 256;
constexpr int TB_THREADS = 1024;
constexpr int TB_BITMAT_MAXD = 1152;
constexpr int TB_BITMAT_HSLOTS = 4096;
constexpr int TB_HASH_MAXD = 8192;

// Dynamic shared memory of one CTA: hash keys + values (hslots), cnt + kc
// (nloc), per warp a segment table and a 64-entry buffer of row indices,
// 4 work words, and R (rows x an odd number of words, to spread the banks).
constexpr int tc_rowstride(int rows) { return ((rows + 31) / 32) | 1; }
constexpr size_t tc_smem(int threads, int hslots, int nloc, int rows) {
    return (size_t)2 * hslots * 4 + (size_t)2 * nloc * 4 + (size_t)(threads / 32) * (sizeof(SegTab) + 128) + 16 +
           (size_t)rows * tc_rowstride(rows) * 4;
}
constexpr size_t TS_SMEM = tc_smem(TS_THREADS, 4 * TS_MAXD, TS_MAXD, TS_MAXD);
constexpr size_t TB_SMEM_BITS = tc_smem(TB_THREADS, TB_BITMAT_HSLOTS, TB_BITMAT_MAXD, TB_BITMAT_MAXD);
constexpr size_t TB_SMEM_HASH = tc_smem(TB_THREADS, 2 * TB_HASH_MAXD, TB_HASH_MAXD, 0);
constexpr size_t TB_SMEM = TB_SMEM_BITS > TB_SMEM_HASH ? TB_SMEM_BITS : TB_SMEM_HASH;
static_assert(TB_SMEM <= 227 * 1024, "k_tri_big shared memory");

__device__ __forceinline__ int out_index(const int *hk, const int *hv, unsigned mask, bool use_hash, const int *ncol,
                                         int s, int e, int w) {
    if (use_hash) return hset_find(hk, hv, mask, w);
    int p = find_sorted(ncol, s, e, w);
    return p < 0 ? -1 : p - s;
}

// One CTA per root u of the list (roots list[0 .. count) or, with BACK,
// list[n - 1], list[n - 2], ...). A root keeps the bit matrix R up to
// bits_maxd and the hash of N+(u) up to hash_maxd (run-time limits no larger
// than the compiled ones, bits_maxd <= hash_maxd), else it probes N+(u) by
// binary search and enumerates the K4 of each triangle.
template <int THREADS, int BITMAT_MAXD, int BITMAT_HSLOTS, int HASH_MAXD, bool BACK, int HMUL>
__device__ __forceinline__ void tri_cta(const Graph &g, int *tcnt, VAcc *vacc, const int *list, int count,
                                        int *next, int bits_maxd, int hash_maxd) {
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int TC_THREADS = THREADS;
    constexpr int NW = THREADS / 32;
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    for (int h = cta_next(next); h < count; h = cta_next(next)) {
        const int u = BACK ? list[g.n - 1 - h] : list[h];
        const int4 ru = g.rinfo[u];
        const int s = ru.y, e = ru.z, dp = e - s;
        const bool use_hash = dp <= HASH_MAXD && dp <= hash_maxd;
        const bool use_bits = use_hash && dp <= BITMAT_MAXD && dp <= bits_maxd;
        unsigned H = use_hash ? next_pow2(HMUL * dp) : 0;   // hash load at most 1 / HMUL, within the carve:
        const unsigned hcap = use_bits ? BITMAT_HSLOTS : 2 * HASH_MAXD;   // its mode's slots
        if (H > hcap) H = hcap;
        const unsigned mask = H ? H - 1 : 0;
        const int W = (dp + 31) >> 5;  // bit-matrix words per row
        const int WP = W | 1;          // row stride of R
        // carve shared memory
        // beyond HASH_MAXD the per-position counters live in global memory
        const int nloc = use_hash ? dp : 0;
        int *hk = reinterpret_cast<int *>(dsm);
        int *hv = hk + H;
        int *cnt = hv + H;
        int *kc = cnt + nloc;
        SegTab *segs = reinterpret_cast<SegTab *>(kc + nloc);   // one per warp
        unsigned short *zb = reinterpret_cast<unsigned short *>(segs + NW) + wid * 64;  // 64 per warp
        int *work = reinterpret_cast<int *>(reinterpret_cast<unsigned short *>(segs + NW) + NW * 64);
        long long *ksum = reinterpret_cast<long long *>(work + 2);    // sum of kc over the rows
        unsigned *R = reinterpret_cast<unsigned *>(work + 4);
        SegTab &seg = segs[wid];
        for (int i = threadIdx.x; i < (int)H; i += TC_THREADS) hk[i] = -1;
        for (int i = threadIdx.x; i < nloc; i += TC_THREADS) { cnt[i] = 0; kc[i] = 0; }
        if (use_bits)
            for (int i = threadIdx.x; i < dp * WP; i += TC_THREADS) R[i] = 0;
        if (threadIdx.x < 4) work[threadIdx.x] = 0;
        __syncthreads();
        if (use_hash)
            for (int i = threadIdx.x; i < dp; i += TC_THREADS) hset_insert(hk, hv, mask, g.ncol[s + i], i);
        const int umax = g.ncol[e - 1];
        __syncthreads();
        long long ku = 0;
        // every warp takes every chunk of 32 out-neighbours and the windows
        // wid, wid + NW, ... of its concatenated lists: no warp waits on a
        // larger chunk of another
        for (int jb = 0; jb < dp - 1; jb += 32) {
            const int j = jb + lane;
            int len = 0, vs = 0;
            if (j < dp - 1) {
                const int4 rv = g.rinfo[g.ncol[s + j]];
                vs = rv.y;
                len = rv.z - rv.y;
            }
            int mypre;
            const int total = seg_build(seg, vs, len, mypre);
            seg_visit<4, true>(g.ncol, seg, mypre, len, total, wid * 32, NW * 32, [&](bool valid, int q, int pos, int w) {
                const int i = (valid && w <= umax) ? out_index(hk, hv, mask, use_hash, g.ncol, s, e, w) : -1;
                const bool hit = i >= 0;
                if (!__any_sync(FULL, hit)) return;
                const int jj = jb + q;
                if (use_bits) {
                    // the upper half of R only; t(u, v) and t(u, w) follow
                    // from R's rows once it is symmetric
                    if (hit) {
                        atomicOr(&R[jj * WP + (i >> 5)], 1u << (i & 31));
                        atomicAdd(&tcnt[pos], 1);
                    }
                    return;
                }
                if (!hit) return;
                atomicAdd(use_hash ? &cnt[jj] : &tcnt[s + jj], 1);
                atomicAdd(use_hash ? &cnt[i] : &tcnt[s + i], 1);
                atomicAdd(&tcnt[pos], 1);
                {
                    // K4 with this triangle (u, v, w): x in N+(w) ∩ N+(u) ∩ N+(v)
                    const int v = g.ncol[s + jj];
                    const int4 rv = g.rinfo[v], rw = g.rinfo[w];
                    const int vs0 = rv.y, ve0 = rv.z;
                    const int ws0 = rw.y, we0 = rw.z;
                    for (int p = ws0; p < we0; ++p) {
                        const int x = g.ncol[p];
                        if (x > umax) break;
                        const int ix = out_index(hk, hv, mask, use_hash, g.ncol, s, e, x);
                        if (ix < 0 || find_sorted(g.ncol, vs0, ve0, x) < 0) continue;
                        ku += 1;
                        if (use_hash) {
                            atomicAdd(&kc[jj], 1);
                            atomicAdd(&kc[i], 1);
                            atomicAdd(&kc[ix], 1);
                        } else {
                            add64(&vacc[v].K4, 1);
                            add64(&vacc[w].K4, 1);
                            add64(&vacc[x].K4, 1);
                        }
                    }
                }
            });
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nloc; i += TC_THREADS)
            if (cnt[i]) atomicAdd(&tcnt[s + i], cnt[i]);
        if (use_bits) {
            // Mirror R: every 32 x 32 block above the diagonal (and the
            // diagonal ones) is transposed by one warp with ballots and ORed
            // into its place below.
            const int nblk = W * (W + 1) / 2;
            for (int bidx = wid; bidx < nblk; bidx += NW) {
                int bj = 0, rem = bidx;
                while (rem >= W - bj) {
                    rem -= W - bj;
                    ++bj;
                }
                const int bi = bj + rem;   // block of rows bj, word bi (bi >= bj)
                const int j = bj * 32 + lane;
                const unsigned wv = j < dp ? R[j * WP + bi] : 0u;
                unsigned tv = 0;
                for (int k = 0; k < 32; ++k) {
                    const unsigned b = __ballot_sync(FULL, (wv >> k) & 1u);
                    if (lane == k) tv = b;
                }
                const int i = bi * 32 + lane;
                if (i < dp) {
                    if (bi == bj) R[i * WP + bj] = wv | tv;
                    else if (tv) R[i * WP + bj] |= tv;
                }
                __syncwarp();
            }
            __syncthreads();
            // K4 credits from the symmetric R: warp per row y, one neighbour
            // z of y per lane, 32 at a time (collected in zb); the row's
            // popcount is t(u, N+(u)[y]) from the triangles rooted at u.
            for (;;) {
                int y = 0;
                if (lane == 0) y = atomicAdd(&work[0], 1);
                y = __shfl_sync(FULL, y, 0);
                if (y >= dp) break;
                const unsigned *ry = R + y * WP;
                long long acc = 0;
                auto batch = [&](int cnt) {
                    if (lane < cnt) {
                        const unsigned *rz = R + zb[lane] * WP;
                        int k = 0;
                        for (int t = 0; t < W; ++t) k += __popc(ry[t] & rz[t]);
                        acc += k;
                    }
                };
                int nb = 0;   // entries waiting in zb (warp-uniform)
                int tuy = 0;  // set bits of row y
                for (int t = 0; t < W; ++t) {
                    const bool set = (ry[t] >> lane) & 1u;
                    const unsigned bal = __ballot_sync(FULL, set);
                    tuy += __popc(bal);
                    if (set) zb[nb + __popc(bal & lanemask_lt())] = (unsigned short)(t * 32 + lane);
                    nb += __popc(bal);
                    __syncwarp();
                    if (nb >= 32) {
                        batch(32);
                        __syncwarp();
                        if (lane < nb - 32) zb[lane] = zb[32 + lane];
                        nb -= 32;
                        __syncwarp();
                    }
                }
                if (nb) batch(nb);
                if (lane == 0 && tuy) atomicAdd(&tcnt[s + y], tuy);
                acc = warp_sum(acc) / 2;   // K4s of u through y
                if (lane == 0 && acc) {
                    kc[y] = (int)acc;
                    atomicAdd((unsigned long long *)ksum, (unsigned long long)acc);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        ku = warp_sum(ku);
        if (lane == 0 && ku) add64(&vacc[u].K4, ku);
        if (use_bits && threadIdx.x == 0 && *ksum) add64(&vacc[u].K4, *ksum / 3);   // each K4 at 3 of N+(u)
        for (int i = threadIdx.x; i < nloc; i += TC_THREADS)
            if (kc[i]) add64(&vacc[g.ncol[s + i]].K4, kc[i]);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(TS_THREADS) k_tri_cta(Graph g, int *tcnt, VAcc *vacc, const int *heavy,
                                                        int *counters, int bits_maxd, int hash_maxd) {
    pdl_begin();
    if (degree_overflow(counters)) return;
    tri_cta<TS_THREADS, TS_MAXD, 4 * TS_MAXD, TS_MAXD, false, 4>(g, tcnt, vacc, heavy, counters[CNT_TRI_HEAVY],
                                                            counters + CNT_TRI_CTA_NEXT, bits_maxd, hash_maxd);
}

__global__ void __launch_bounds__(TB_THREADS) k_tri_big(Graph g, int *tcnt, VAcc *vacc, const int *heavy,
                                                        int *counters, int bits_maxd, int hash_maxd) {
    pdl_begin();
    if (degree_overflow(counters)) return;
    tri_cta<TB_THREADS, TB_BITMAT_MAXD, TB_BITMAT_HSLOTS, TB_HASH_MAXD, true, 4>(g, tcnt, vacc, heavy,
                                                                            counters[CNT_TRI_BIG],
                                                                            counters + CNT_TRI_BIG_NEXT, bits_maxd,
                                                                            hash_maxd);
}


void launch_stage1(Work &w, cudaStream_t st) {
    Graph g{w.n, w.m, w.rinfo, w.ncol};
    const int maxd = w.tune[TUNE_WARP_MAXD] < TW_MAXD ? w.tune[TUNE_WARP_MAXD] : TW_MAXD;
    static const int occ_w = resident_ctas((const void *)k_tri_warp, TW_WARPS * 32, 0);
    static const int occ_c = resident_ctas((const void *)k_tri_cta, TS_THREADS, TS_SMEM);
    static const int occ_b = resident_ctas((const void *)k_tri_big, TB_THREADS, TB_SMEM);
    launch_pdl(k_tri_warp, w.num_sms * min(w.tune[TUNE_GRID_TRI], occ_w), TW_WARPS * 32, 0, st, g, w.tcnt, w.vacc, w.lists,
                                                                                       w.counters, maxd);
    after_launch(st, K_TRI_WARP);
    const int bits = w.tune[TUNE_TRI_BITS_MAXD], hash = w.tune[TUNE_TRI_HASH_MAXD];
    launch_pdl(k_tri_cta, w.num_sms * occ_c, TS_THREADS, TS_SMEM, st, g, w.tcnt, w.vacc, w.lists, w.counters, bits, hash);
    after_launch(st, K_TRI_CTA);
    launch_pdl(k_tri_big, w.num_sms * occ_b, TB_THREADS, TB_SMEM, st, g, w.tcnt, w.vacc, w.lists, w.counters, bits, hash);
    after_launch(st, K_TRI_BIG);
}

void configure_stage1() {
    cudaFuncSetAttribute(k_tri_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS_SMEM);
    cudaFuncSetAttribute(k_tri_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TB_SMEM);
}

}  // namespace niorca
