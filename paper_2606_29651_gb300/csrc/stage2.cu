// stage2.cu -- edge aggregates and the triangle-opposite term, after the
// per-edge triangle counts t are final.
//
// For every out-edge (u, v) with t = t_uv > 0 (edges without a triangle add
// nothing), both endpoints receive
//   A1 += t, A2 += t^2, A3 += t * d(other end),
// the neighbour sums from which the f* variables of Table 1 that involve
// t_xy follow (f_13^14 = A2 - A1, f_11^13 = (d-1) A1 - A2, ...).
// Every triangle u < v < w is listed again (as in Stage I) and each corner
// receives t of the opposite edge minus one:
//   D12[u] += t_vw - 1, D12[v] += t_uw - 1, D12[w] += t_uv - 1,
// so that D12(x) = sum over triangles {x,y,z} of (t_yz - 1) = f_12^14
// (Table 1: the triangles of e_yz other than xyz). Only out-edges with
// t > 0 are expanded.
#include "kernels.h"

namespace niorca {

constexpr int AW_MAXD = 64;
constexpr int AW_WARPS = 8;
constexpr int AS_MAXD = 256;   // out-degree handled by a 256-thread CTA (k_agg_cta)

struct __align__(16) AggWarpSmem {
    int hk[4 * AW_MAXD];   // N+(u) hash at load <= 1/4 (most probes are misses)
    int hv[4 * AW_MAXD];
    long long dc[AW_MAXD];
    SegTab seg;
};

// Edge aggregates of u's out-edges; returns whether any has a triangle.
__device__ __forceinline__ bool edge_aggregates(const Graph &g, const int *tcnt, VAcc *vacc, int u, int s, int dp,
                                                int first, int stride) {
    const int4 ru = g.rinfo[u];
    const int du = ru.z - ru.x;
    long long a1 = 0, a2 = 0, a3 = 0;
    for (int j = first; j < dp; j += stride) {
        const long long t = tcnt[s + j];
        if (!t) continue;
        const int v = g.ncol[s + j];
        const int4 rv = g.rinfo[v];
        const long long dv = rv.z - rv.x;
        a1 += t;
        a2 += t * t;
        a3 += t * dv;
        add64(&vacc[v].A1, t);
        add64(&vacc[v].A2, t * t);
        add64(&vacc[v].A3, t * du);
    }
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    a3 = warp_sum(a3);
    if (lane_id() == 0 && a1) {
        add64(&vacc[u].A1, a1);
        add64(&vacc[u].A2, a2);
        add64(&vacc[u].A3, a3);
    }
    return a1 != 0;
}

__global__ void __launch_bounds__(AW_WARPS * 32, 8) k_agg_warp(Graph g, const int *tcnt, VAcc *vacc, int *heavy,
                                                            int *counters, int maxd) {
    pdl_begin();
    __shared__ AggWarpSmem sm_all[AW_WARPS];
    AggWarpSmem &S = sm_all[threadIdx.x >> 5];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (degree_overflow(counters)) return;
    for (int u = gw; u < g.n; u += nw) {
        const int4 ru = g.rinfo[u];
        const int s = ru.y, e = ru.z, dp = e - s;
        if (dp < 1) continue;
        if (dp > maxd) {
            if (lane == 0) {
                if (dp <= AS_MAXD) heavy[atomicAdd(&counters[CNT_AGG_HEAVY], 1)] = u;
                else heavy[g.n - 1 - atomicAdd(&counters[CNT_AGG_BIG], 1)] = u;
            }
            continue;
        }
        if (!edge_aggregates(g, tcnt, vacc, u, s, dp, lane, 32) || dp < 2) continue;
        const unsigned mask = next_pow2(4 * dp) - 1;
        for (int i = lane; i <= (int)mask; i += 32) S.hk[i] = -1;
        for (int i = lane; i < AW_MAXD; i += 32) S.dc[i] = 0;
        __syncwarp();
        for (int i = lane; i < dp; i += 32) hset_insert(S.hk, S.hv, mask, g.ncol[s + i], i);
        const int umax = g.ncol[e - 1];
        __syncwarp();
        long long du12 = 0;
        for (int jb = 0; jb < dp - 1; jb += 32) {
            const int j = jb + lane;
            int len = 0, vs = 0;
            if (j < dp - 1 && tcnt[s + j] > 0) {
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
                if (!hit) return;
                add64(&S.dc[jj], tcnt[s + i] - 1);                           // t(u, w) - 1 -> v
                du12 += tcnt[pos] - 1;                                       // t(v, w) - 1 -> u
                atomicAdd((unsigned long long *)&S.dc[i], (unsigned long long)(tcnt[s + jj] - 1));  // t(u, v) - 1 -> w
            });
            __syncwarp();
        }
        du12 = warp_sum(du12);
        if (lane == 0 && du12) add64(&vacc[u].D12, du12);
        for (int i = lane; i < dp; i += 32)
            if (S.dc[i]) add64(&vacc[g.ncol[s + i]].D12, S.dc[i]);
        __syncwarp();
    }
}

// Roots above the warp tier: k_agg_cta (256 threads, dp <= AS_MAXD, about
// 21 KB of shared memory, several CTAs per SM) and k_agg_big (1024 threads),
// from the front and the back of the heavy list. Up to AB_BITMAT_MAXD the
// triangles of u are kept as the upper half of a bit matrix R of N+(u) (as
// in Stage I): a hit sets its bit and adds t(v, w) - 1 to u; R is then made
// symmetric, and each y in N+(u) receives the sum over its neighbours z in
// R of t(u, z) - 1 (t(u, .) cached in shared memory). Above that, a hash of
// N+(u) up to AB_HASH_MAXD and per-triangle credits; binary searches beyond.
constexpr int AS_THREADS = 256;
constexpr int AB_THREADS = 1024;
constexpr int AB_BITMAT_MAXD = 1152;
constexpr int AB_BITMAT_HSLOTS = 4096;
constexpr int AB_HASH_MAXD = 8192;
constexpr int ac_rowstride(int rows) { return ((rows + 31) / 32) | 1; }
// dc (nloc x 8 B, hash-only mode), hash (2 x hslots ints), t(u, .) cache
// (rows ints), per warp a segment table and 64 row indices, 4 work words, R.
constexpr size_t ac_smem(int threads, int hslots, int nloc, int rows) {
    return (size_t)nloc * 8 + (size_t)2 * hslots * 4 + (size_t)rows * 4 + (size_t)(threads / 32) * (sizeof(SegTab) + 128) +
           16 + (size_t)rows * ac_rowstride(rows) * 4;
}
constexpr size_t AS_SMEM = ac_smem(AS_THREADS, 4 * AS_MAXD, 0, AS_MAXD);
constexpr size_t AB_SMEM_BITS = ac_smem(AB_THREADS, AB_BITMAT_HSLOTS, 0, AB_BITMAT_MAXD);
constexpr size_t AB_SMEM_HASH = ac_smem(AB_THREADS, 2 * AB_HASH_MAXD, AB_HASH_MAXD, 0);
constexpr size_t AB_SMEM = AB_SMEM_BITS > AB_SMEM_HASH ? AB_SMEM_BITS : AB_SMEM_HASH;
static_assert(AB_SMEM <= 227 * 1024, "k_agg_big shared memory");

template <int THREADS, int BITMAT_MAXD, int BITMAT_HSLOTS, int HASH_MAXD, bool BACK, int HMUL>
__device__ __forceinline__ void agg_cta(const Graph &g, const int *tcnt, VAcc *vacc, const int *heavy, int nh,
                                        int *next, int bits_maxd, int hash_maxd) {
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int NW = THREADS / 32;
    __shared__ int any_tri;
    const int lane = lane_id(), wid = threadIdx.x >> 5;
    for (int h = cta_next(next); h < nh; h = cta_next(next)) {
        const int u = BACK ? heavy[g.n - 1 - h] : heavy[h];
        const int4 ru = g.rinfo[u];
        const int s = ru.y, e = ru.z, dp = e - s;
        if (threadIdx.x == 0) any_tri = 0;
        __syncthreads();
        if (edge_aggregates(g, tcnt, vacc, u, s, dp, threadIdx.x, THREADS) && lane == 0) any_tri = 1;
        __syncthreads();
        if (!any_tri) continue;
        const bool use_hash = dp <= HASH_MAXD && dp <= hash_maxd;
        const bool use_bits = use_hash && dp <= BITMAT_MAXD && dp <= bits_maxd;
        unsigned H = use_hash ? next_pow2(HMUL * dp) : 0;   // hash load at most 1 / HMUL, within the carve:
        const unsigned hcap = use_bits ? BITMAT_HSLOTS : 2 * HASH_MAXD;   // its mode's slots
        if (H > hcap) H = hcap;
        const unsigned mask = H ? H - 1 : 0;
        const int W = (dp + 31) >> 5, WP = W | 1;   // words per row of R, row stride
        const int nloc = (use_hash && !use_bits) ? dp : 0;
        const int nrow = use_bits ? dp : 0;
        long long *dc = reinterpret_cast<long long *>(dsm);   // hash-only mode
        int *hk = reinterpret_cast<int *>(dc + ((nloc + 1) & ~1));   // 16-byte aligned buckets
        int *hv = hk + H;
        int *T = hv + H;                                       // t(u, N+(u)[i]), bit-matrix mode
        SegTab *segs = reinterpret_cast<SegTab *>(T + nrow);
        int *work = reinterpret_cast<int *>(reinterpret_cast<unsigned short *>(segs + NW) + NW * 64);
        unsigned *R = reinterpret_cast<unsigned *>(work + 4);
        SegTab &seg = segs[wid];
        for (int i = threadIdx.x; i < (int)H; i += THREADS) hk[i] = -1;
        for (int i = threadIdx.x; i < nloc; i += THREADS) dc[i] = 0;
        for (int i = threadIdx.x; i < nrow; i += THREADS) T[i] = tcnt[s + i];
        if (use_bits)
            for (int i = threadIdx.x; i < dp * WP; i += THREADS) R[i] = 0;
        if (threadIdx.x < 4) work[threadIdx.x] = 0;
        __syncthreads();
        if (use_hash)
            for (int i = threadIdx.x; i < dp; i += THREADS) hset_insert(hk, hv, mask, g.ncol[s + i], i);
        const int umax = g.ncol[e - 1];
        __syncthreads();
        long long du12 = 0;
        for (int jb = 0; jb < dp - 1; jb += 32) {   // all warps share each chunk
            const int j = jb + lane;
            int len = 0, vs = 0;
            if (j < dp - 1 && tcnt[s + j] > 0) {
                const int4 rv = g.rinfo[g.ncol[s + j]];
                vs = rv.y;
                len = rv.z - rv.y;
            }
            int mypre;
            const int total = seg_build(seg, vs, len, mypre);
            seg_visit<4, true>(g.ncol, seg, mypre, len, total, wid * 32, NW * 32, [&](bool valid, int q, int pos, int w) {
                int i = -1;
                if (valid && w <= umax) {
                    if (use_hash) {
                        i = hset_find(hk, hv, mask, w);
                    } else {
                        const int p = find_sorted(g.ncol, s, e, w);
                        i = p < 0 ? -1 : p - s;
                    }
                }
                const bool hit = i >= 0;
                if (!__any_sync(FULL, hit)) return;
                const int jj = jb + q;
                if (hit) du12 += tcnt[pos] - 1;   // t(v, w) - 1 -> u
                if (use_bits) {
                    if (hit) atomicOr(&R[jj * WP + (i >> 5)], 1u << (i & 31));
                    return;
                }
                if (!hit) return;
                add64(use_hash ? &dc[jj] : &vacc[g.ncol[s + jj]].D12, tcnt[s + i] - 1);   // t(u, w) - 1 -> v
                const long long tw = tcnt[s + jj] - 1;                                      // t(u, v) - 1 -> w
                if (use_hash) atomicAdd((unsigned long long *)&dc[i], (unsigned long long)tw);
                else add64(&vacc[w].D12, tw);
            });
            __syncwarp();
        }
        __syncthreads();
        du12 = warp_sum(du12);
        if (lane == 0 && du12) add64(&vacc[u].D12, du12);
        if (use_bits) {
            // mirror R (a ballot transpose per 32 x 32 block), then y in N+(u)
            // receives the sum over its neighbours z in R of t(u, z) - 1
            const int nblk = W * (W + 1) / 2;
            for (int bidx = wid; bidx < nblk; bidx += NW) {
                int bj = 0, rem = bidx;
                while (rem >= W - bj) {
                    rem -= W - bj;
                    ++bj;
                }
                const int bi = bj + rem;
                const int jr = bj * 32 + lane;
                const unsigned wv = jr < dp ? R[jr * WP + bi] : 0u;
                unsigned tv = 0;
                for (int k = 0; k < 32; ++k) {
                    const unsigned b = __ballot_sync(FULL, (wv >> k) & 1u);
                    if (lane == k) tv = b;
                }
                const int ir = bi * 32 + lane;
                if (ir < dp) {
                    if (bi == bj) R[ir * WP + bj] = wv | tv;
                    else if (tv) R[ir * WP + bj] |= tv;
                }
                __syncwarp();
            }
            __syncthreads();
            for (int y = wid; y < dp; y += NW) {
                const unsigned *ry = R + y * WP;
                long long c = 0;
                for (int t = 0; t < W; ++t) {
                    const int z = t * 32 + lane;
                    if ((ry[t] >> lane) & 1u) c += T[z] - 1;
                }
                c = warp_sum(c);
                if (lane == 0 && c) add64(&vacc[g.ncol[s + y]].D12, c);
            }
        }
        for (int i = threadIdx.x; i < nloc; i += THREADS)
            if (dc[i]) add64(&vacc[g.ncol[s + i]].D12, dc[i]);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(AS_THREADS) k_agg_cta(Graph g, const int *tcnt, VAcc *vacc, const int *heavy,
                                                        int *counters, int bits_maxd, int hash_maxd) {
    pdl_begin();
    if (degree_overflow(counters)) return;
    agg_cta<AS_THREADS, AS_MAXD, 4 * AS_MAXD, AS_MAXD, false, 4>(g, tcnt, vacc, heavy, counters[CNT_AGG_HEAVY],
                                                            counters + CNT_AGG_CTA_NEXT, bits_maxd, hash_maxd);
}

__global__ void __launch_bounds__(AB_THREADS) k_agg_big(Graph g, const int *tcnt, VAcc *vacc, const int *heavy,
                                                        int *counters, int bits_maxd, int hash_maxd) {
    pdl_begin();
    if (degree_overflow(counters)) return;
    agg_cta<AB_THREADS, AB_BITMAT_MAXD, AB_BITMAT_HSLOTS, AB_HASH_MAXD, true, 4>(g, tcnt, vacc, heavy,
                                                                            counters[CNT_AGG_BIG],
                                                                            counters + CNT_AGG_BIG_NEXT, bits_maxd,
                                                                            hash_maxd);
}

void launch_stage2(Work &w, cudaStream_t st) {
    Graph g{w.n, w.m, w.rinfo, w.ncol};
    int *heavy = w.lists + (size_t)w.n;
    const int maxd = w.tune[TUNE_WARP_MAXD] < AW_MAXD ? w.tune[TUNE_WARP_MAXD] : AW_MAXD;
    static const int occ_w = resident_ctas((const void *)k_agg_warp, AW_WARPS * 32, 0);
    static const int occ_c = resident_ctas((const void *)k_agg_cta, AS_THREADS, AS_SMEM);
    static const int occ_b = resident_ctas((const void *)k_agg_big, AB_THREADS, AB_SMEM);
    launch_pdl(k_agg_warp, w.num_sms * min(w.tune[TUNE_GRID_AGG], occ_w), AW_WARPS * 32, 0, st, g, w.tcnt, w.vacc, heavy,
                                                                                       w.counters, maxd);
    after_launch(st, K_AGG_WARP);
    const int bits = w.tune[TUNE_TRI_BITS_MAXD], hash = w.tune[TUNE_TRI_HASH_MAXD];
    launch_pdl(k_agg_cta, w.num_sms * occ_c, AS_THREADS, AS_SMEM, st, g, w.tcnt, w.vacc, heavy, w.counters, bits, hash);
    after_launch(st, K_AGG_CTA);
    launch_pdl(k_agg_big, w.num_sms * occ_b, AB_THREADS, AB_SMEM, st, g, w.tcnt, w.vacc, heavy, w.counters, bits, hash);
    after_launch(st, K_AGG_BIG);
}

void configure_stage2() {
    cudaFuncSetAttribute(k_agg_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AS_SMEM);
    cudaFuncSetAttribute(k_agg_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AB_SMEM);
}

}  // namespace niorca
