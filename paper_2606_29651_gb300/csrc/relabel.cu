// relabel.cu -- degree-ordered relabelling of the input CSR.
//
// Algorithm 2 orients every edge from the smaller to the larger vertex id
// (y.id > x.id) so that each triangle and each K4 is found once. Any total
// order keeps that property; this implementation uses (degree class, id),
// with four classes per octave of degree, so that the out-lists of the
// oriented graph stay short on skewed graphs (a hub only points at other
// hubs). Vertices are renumbered in that order; in the relabelled CSR every
// row is ascending, so N+(u) = {v in N(u): v > u} is the suffix of row u
// starting at split[u], and N-(u) is the prefix.
//
// Because new ids inside one class follow old ids, a row of the input that
// is sorted by old id becomes sorted by new id after a stable partition by
// class: no sort is needed, only per-class counting.
#include "kernels.h"

namespace niorca {

// ------------------------------------------------------------ exclusive scan

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_THREAD = SCAN_TILE / SCAN_THREADS;

size_t scan_partials(long long len) { return (size_t)((len + SCAN_TILE - 1) / SCAN_TILE) + 1; }

__device__ __forceinline__ int block_exclusive_scan(int v, int *wsum, int *total) {
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = warp_inclusive_scan(v);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < nw ? wsum[lane] : 0;
        int xi = warp_inclusive_scan(x);
        if (lane < nw) wsum[lane] = xi - x;
        if (lane == nw - 1) *total = xi;
    }
    __syncthreads();
    int r = incl - v + wsum[w];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int *in, long long len, int *part) {
    pdl_begin();
    __shared__ int wsum[32];
    __shared__ int tot;
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    int s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        long long g = base + i;
        if (g < len) s += in[g];
    }
    block_exclusive_scan(s, wsum, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(int *part, int nblocks) {
    pdl_begin();
    __shared__ int wsum[32];
    __shared__ int tot;
    int carry = 0;
    for (int b0 = 0; b0 < nblocks; b0 += 1024) {
        int i = b0 + threadIdx.x;
        int v = i < nblocks ? part[i] : 0;
        int ex = block_exclusive_scan(v, wsum, &tot);
        if (i < nblocks) part[i] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nblocks] = carry;
}

// With part == nullptr a single block scans the whole array (len <= SCAN_TILE).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const int *in, int *out, long long len, const int *part,
                                                           int write_total) {
    pdl_begin();
    __shared__ int tile[SCAN_TILE];
    __shared__ int wsum[32];
    __shared__ int tot;
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        long long g = base + i;
        tile[i] = g < len ? in[g] : 0;
    }
    __syncthreads();
    int local[SCAN_PER_THREAD];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        local[k] = tile[threadIdx.x * SCAN_PER_THREAD + k];
        s += local[k];
    }
    int ex = block_exclusive_scan(s, wsum, &tot) + (part ? part[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        tile[threadIdx.x * SCAN_PER_THREAD + k] = ex;
        ex += local[k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        long long g = base + i;
        if (g < len) out[g] = tile[i];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[len] = part ? part[gridDim.x] : tot;
}

void launch_exclusive_scan(const int *in, int *out, long long len, bool write_total, int *part,
                           cudaStream_t st) {
    const int nb = (int)((len + SCAN_TILE - 1) / SCAN_TILE);
    if (nb == 0) {
        if (write_total) cudaMemsetAsync(out, 0, sizeof(int), st);
        return;
    }
    if (nb == 1) {   // one tile: one launch
        launch_pdl(k_scan_down, 1, SCAN_THREADS, 0, st, in, out, len, nullptr, write_total ? 1 : 0);
        after_launch(st, K_SCAN);
        return;
    }
    launch_pdl(k_scan_reduce, nb, SCAN_THREADS, 0, st, in, len, part);
    after_launch(st, K_SCAN);
    launch_pdl(k_scan_top, 1, 1024, 0, st, part, nb);
    after_launch(st, K_SCAN);
    launch_pdl(k_scan_down, nb, SCAN_THREADS, 0, st, in, out, len, part, write_total ? 1 : 0);
    after_launch(st, K_SCAN);
}

// ------------------------------------------------------------- class order

constexpr int RL_THREADS = 256;

// Degrees (with offset validation) and the class histogram of each tile.
__global__ void __launch_bounds__(RL_THREADS) k_class_hist(const int *rowptr, int n, int m, int2 *vinfo, int *chist,
                                                           int ntiles, int *counters, int *status) {
    pdl_begin();
    __shared__ int h[NCLASS];
    __shared__ int smax;
    for (int c = threadIdx.x; c < NCLASS; c += RL_THREADS) h[c] = 0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    int lmax = 0, bad = 0;
    const int tile = blockIdx.x;
    for (int i = threadIdx.x; i < RL_TILE; i += RL_THREADS) {
        const long long x = (long long)tile * RL_TILE + i;
        if (x >= n) break;
        const int a = rowptr[x], b = rowptr[x + 1];
        const bool ok = a >= 0 && b >= a && b <= m;
        const int d = ok ? b - a : 0;
        if (!ok || (x == 0 && a != 0) || (x == n - 1 && b != m)) bad = 1;
        vinfo[x] = make_int2(-1, d);
        atomicAdd(&h[deg_class(d)], 1);
        lmax = max(lmax, d);
    }
    if (bad) set_status(status, ST_EINVAL);
    lmax = warp_max(lmax);
    if (lane_id() == 0) atomicMax(&smax, lmax);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&counters[CNT_DMAX], smax);
        if (smax > MAX_DEGREE) set_status(status, ST_EOVERFLOW);
    }
    for (int c = threadIdx.x; c < NCLASS; c += RL_THREADS) chist[c * ntiles + tile] = h[c];
}

// New id of every vertex: class offset + stable rank by old id within class.
__global__ void __launch_bounds__(RL_THREADS) k_class_scatter(int n, int2 *vinfo, const int *coff, int ntiles,
                                                              int *perm, int *ndeg) {
    pdl_begin();
    constexpr int NW = RL_THREADS / 32;
    __shared__ int run[NCLASS];
    __shared__ int tot[NCLASS];
    __shared__ int wc[NW][NCLASS];
    const int tile = blockIdx.x, lane = lane_id(), w = threadIdx.x >> 5;
    for (int c = threadIdx.x; c < NCLASS; c += RL_THREADS) run[c] = 0;
    for (int k = 0; k < RL_TILE / RL_THREADS; ++k) {
        for (int i = threadIdx.x; i < NW * NCLASS; i += RL_THREADS) (&wc[0][0])[i] = 0;
        __syncthreads();
        const long long x = (long long)tile * RL_TILE + k * RL_THREADS + threadIdx.x;
        const bool valid = x < n;
        const int d = valid ? vinfo[x].y : 0;
        const int c = valid ? deg_class(d) : NCLASS + lane;  // invalid lanes match only themselves
        const unsigned peers = __match_any_sync(FULL, c);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wc[w][c] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < NCLASS) {
            int s = 0;
            for (int ww = 0; ww < NW; ++ww) {
                int t = wc[ww][threadIdx.x];
                wc[ww][threadIdx.x] = s;
                s += t;
            }
            tot[threadIdx.x] = s;
        }
        __syncthreads();
        if (valid) {
            const int id = coff[c * ntiles + tile] + run[c] + wc[w][c] + rank;
            vinfo[x].x = id;
            perm[id] = (int)x;
            ndeg[id] = d;
        }
        __syncthreads();
        if (threadIdx.x < NCLASS) run[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
}

// The class order of a graph of at most RL_TILE vertices in one CTA, with no
// launch in between: the degree pass and class histogram of k_class_hist,
// the scan of the class offsets, the stable class scatter of k_class_scatter
// and the scan of the new degrees into the new row offsets (nrow[n] = m).
constexpr int RS_THREADS = 1024;
__global__ void __launch_bounds__(RS_THREADS) k_class_small(const int *rowptr, int n, int m, int2 *vinfo, int *coff,
                                                            int *perm, int *nrow, int *counters, int *status) {
    pdl_begin();
    constexpr int NW = RS_THREADS / 32;
    __shared__ int h[NCLASS];          // class counts, then each class's next id
    __shared__ int wc[NW][NCLASS];     // per-warp class counts, then offsets
    __shared__ int deg[RL_TILE];       // degree of each vertex
    __shared__ int nd[RL_TILE];        // degree of each new id
    __shared__ int wsum[32];
    __shared__ int tot, smax;
    const int lane = lane_id(), w = threadIdx.x >> 5;
    for (int c = threadIdx.x; c < NCLASS; c += RS_THREADS) h[c] = 0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    int lmax = 0, bad = 0;
    for (int x = threadIdx.x; x < n; x += RS_THREADS) {
        const int a = rowptr[x], b = rowptr[x + 1];
        const bool ok = a >= 0 && b >= a && b <= m;
        const int d = ok ? b - a : 0;
        if (!ok || (x == 0 && a != 0) || (x == n - 1 && b != m)) bad = 1;
        deg[x] = d;
        atomicAdd(&h[deg_class(d)], 1);
        lmax = max(lmax, d);
    }
    if (bad) set_status(status, ST_EINVAL);
    lmax = warp_max(lmax);
    if (lane == 0) atomicMax(&smax, lmax);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&counters[CNT_DMAX], smax);
        if (smax > MAX_DEGREE) set_status(status, ST_EOVERFLOW);
    }
    {   // class offsets (NCLASS <= RS_THREADS)
        const int ex = block_exclusive_scan(threadIdx.x < NCLASS ? h[threadIdx.x] : 0, wsum, &tot);
        if (threadIdx.x < NCLASS) {
            h[threadIdx.x] = ex;
            coff[threadIdx.x] = ex;
        }
    }
    // new ids: stable rank by old id within the class, RS_THREADS vertices at a time
    for (int x0 = 0; x0 < n; x0 += RS_THREADS) {
        for (int i = threadIdx.x; i < NW * NCLASS; i += RS_THREADS) (&wc[0][0])[i] = 0;
        __syncthreads();
        const int x = x0 + threadIdx.x;
        const bool valid = x < n;
        const int d = valid ? deg[x] : 0;
        const int c = valid ? deg_class(d) : NCLASS + lane;   // invalid lanes match only themselves
        const unsigned peers = __match_any_sync(FULL, c);
        const int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wc[w][c] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < NCLASS) {
            int run = h[threadIdx.x];
            for (int ww = 0; ww < NW; ++ww) {
                const int t = wc[ww][threadIdx.x];
                wc[ww][threadIdx.x] = run;
                run += t;
            }
            h[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const int id = wc[w][c] + rank;
            vinfo[x] = make_int2(id, d);
            perm[id] = x;
            nd[id] = d;
        }
        __syncthreads();
    }
    int carry = 0;   // new row offsets
    for (int i0 = 0; i0 < n; i0 += RS_THREADS) {
        const int i = i0 + threadIdx.x;
        const int ex = block_exclusive_scan(i < n ? nd[i] : 0, wsum, &tot);
        if (i < n) nrow[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) nrow[n] = carry;
}

// Union id of a column entry: graphs of a batch store ids local to the graph,
// whose vertices occupy [vr.x, vr.y) of the union; -1 if out of range.
__device__ __forceinline__ int global_id(int y, int2 vr, int n) {
    const long long g = (long long)vr.x + y;
    return (y >= 0 && g < vr.y && g >= 0 && g < n) ? (int)g : -1;
}

__device__ __forceinline__ long long c2m1(int d) {  // C(d - 1, 2)
    long long a = d - 1;
    return a * (a - 1) / 2;
}

// Row relabelling, one warp per row (rows below LONG_ROW_CLASS), taken in
// input order so that the rows are read sequentially and written scattered.
// Pass 1 validates the row, counts its classes and sums neighbour degrees;
// pass 2 writes every new id at its class offset (stable within a class);
// the first 64 entries keep their new id and class in registers between
// the passes.
__global__ void __launch_bounds__(256) k_relabel_rows_warp(const int *rowptr, const int *colidx, int n,
                                                           const int2 *vrange, const int2 *vinfo, const int *perm,
                                                           const int *nrow, const int *coff, int ntiles, int *ncol,
                                                           int4 *rinfo, VAcc *vacc, int *tcnt, int *status,
                                                           int long_class) {
    pdl_begin();
    __shared__ int hist_all[8][NCLASS];
    const int lane = lane_id();
    int *H = hist_all[threadIdx.x >> 5];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int bad = 0;
    for (int x = gw; x < n; x += nw) {
        const int2 vx = vinfo[x];   // new id, degree (0 for a row with bad offsets)
        const int r = vx.x, d = vx.y;
        if (deg_class(d) >= long_class) continue;   // a CTA takes it
        const int ob = d > 0 ? rowptr[x] : 0;
        const int nb = nrow[r];
        const int2 vr = vrange ? vrange[x] : make_int2(0, n);
        if (d <= 32) {
            // One entry per lane: its place in the relabelled row is the
            // number of entries of a lower class plus those of its class
            // before it, from eight ballots over the class bits (inactive
            // lanes take class NCLASS, above every real one).
            const bool act = lane < d;
            const int y = act ? colidx[ob + lane] : 0;
            const int yp = __shfl_up_sync(FULL, y, 1);
            int nid = 0, c = NCLASS;
            unsigned dl = 0, bl = 0;
            long long p6l = 0;
            if (act) {
                int ys = global_id(y, vr, n);
                if (ys < 0) { bad |= ST_EINVAL; ys = x; }
                else if (ys == x || (lane > 0 && y <= yp)) bad |= ST_ENOTSIMPLE;
                const int2 vi = vinfo[ys];
                nid = vi.x;
                c = deg_class(vi.y);
                dl = (unsigned)vi.y;
                p6l = c2m1(vi.y);
                bl = vi.x < r;
            }
            static_assert(NCLASS < 256, "classes and the inactive value NCLASS fit eight bits");
            unsigned eq = FULL, lt = 0;
#pragma unroll
            for (int bit = 7; bit >= 0; --bit) {
                const bool one = (c >> bit) & 1;
                const unsigned ones = __ballot_sync(FULL, one);
                if (one) {
                    lt |= eq & ~ones;
                    eq &= ones;
                } else {
                    eq &= ~ones;
                }
            }
            if (act) ncol[nb + __popc(lt) + __popc(eq & lanemask_lt())] = nid;
            // neighbour degrees are at most MAX_DEGREE: 32 of them fit 32 bits
            const long long s1 = __reduce_add_sync(FULL, dl);
            const int below = (int)__reduce_add_sync(FULL, bl);
            const long long p6 = warp_sum(p6l);
            const int sp = nb + below;
            if (lane == 0) {
                rinfo[r] = make_int4(nb, sp, nb + d, 0);
                VAcc a;
                a.S1 = s1; a.A1 = 0; a.P6 = p6; a.A2 = 0; a.A3 = 0; a.D12 = 0; a.K4 = 0; a.C4 = 0;
                vacc[r] = a;
            }
            if (sp + lane < nb + d) tcnt[sp + lane] = 0;
            continue;
        }
        for (int c = lane; c < NCLASS; c += 32) H[c] = 0;
        __syncwarp();
        long long s1 = 0, p6 = 0;
        int below = 0, last = -1;
        int nv0 = 0, nc0 = NCLASS + lane, nv1 = 0, nc1 = NCLASS + lane;   // entries lane and 32 + lane
        for (int k = 0; k < d; k += 32) {
            const int i = k + lane;
            const bool act = i < d;
            const int y = act ? colidx[ob + i] : 0;
            int yp = __shfl_up_sync(FULL, y, 1);
            if (lane == 0) yp = last;
            last = __shfl_sync(FULL, y, 31);
            if (act) {
                int ys = global_id(y, vr, n);
                if (ys < 0) { bad |= ST_EINVAL; ys = x; }
                else if (ys == x || (i > 0 && y <= yp)) bad |= ST_ENOTSIMPLE;
                const int2 vi = vinfo[ys];
                const int c = deg_class(vi.y);
                atomicAdd(&H[c], 1);
                s1 += vi.y;
                p6 += c2m1(vi.y);
                below += vi.x < r;
                if (k == 0) { nv0 = vi.x; nc0 = c; }
                else if (k == 32) { nv1 = vi.x; nc1 = c; }
            }
        }
        // exclusive scan of the 128 class counts: 4 per lane
        __syncwarp();
        {
            int a0 = H[4 * lane], a1 = H[4 * lane + 1], a2 = H[4 * lane + 2], a3 = H[4 * lane + 3];
            int sum = a0 + a1 + a2 + a3;
            int ex = warp_inclusive_scan(sum) - sum;
            H[4 * lane] = ex;
            H[4 * lane + 1] = ex + a0;
            H[4 * lane + 2] = ex + a0 + a1;
            H[4 * lane + 3] = ex + a0 + a1 + a2;
        }
        __syncwarp();
        for (int k = 0; k < d; k += 32) {
            const int i = k + lane;
            const bool act = i < d;
            int nid, c;
            if (k == 0) { nid = nv0; c = nc0; }
            else if (k == 32) { nid = nv1; c = nc1; }
            else {
                int ys = act ? global_id(colidx[ob + i], vr, n) : 0;
                if (ys < 0) ys = x;
                const int2 vi = act ? vinfo[ys] : make_int2(0, 0);
                nid = vi.x;
                c = act ? deg_class(vi.y) : NCLASS + lane;
            }
            const unsigned peers = __match_any_sync(FULL, c);
            const int rank = __popc(peers & lanemask_lt());
            int pos = 0;
            if (act) pos = H[c] + rank;
            __syncwarp();
            if (act && rank == 0) H[c] += __popc(peers);
            __syncwarp();
            if (act) ncol[nb + pos] = nid;
        }
        s1 = warp_sum(s1);
        p6 = warp_sum(p6);
        below = warp_sum(below);
        const int sp = nb + below;
        if (lane == 0) {
            rinfo[r] = make_int4(nb, sp, nb + d, 0);
            VAcc a;
            a.S1 = s1; a.A1 = 0; a.P6 = p6; a.A2 = 0; a.A3 = 0; a.D12 = 0; a.K4 = 0; a.C4 = 0;
            vacc[r] = a;
        }
        for (int p = sp + lane; p < nb + d; p += 32) tcnt[p] = 0;
        __syncwarp();
    }
    bad = __reduce_or_sync(FULL, bad);
    if (lane == 0 && bad) set_status(status, bad);
}

// Row relabelling, one CTA per long row (rows from LONG_ROW_CLASS on).
constexpr int RLC_THREADS = 512;
__global__ void __launch_bounds__(RLC_THREADS) k_relabel_rows_cta(const int *rowptr, const int *colidx, int n,
                                                                  const int2 *vrange, const int2 *vinfo,
                                                                  const int *perm,
                                                                  const int *nrow, const int *coff, int ntiles,
                                                                  int *ncol, int4 *rinfo, VAcc *vacc, int *tcnt,
                                                                  int *status, int long_class) {
    pdl_begin();
    constexpr int NW = RLC_THREADS / 32;
    __shared__ int H[NCLASS];
    __shared__ int tot[NCLASS];
    __shared__ int wc[NW][NCLASS];
    __shared__ long long red[3][NW];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int bound = coff[long_class * ntiles];
    int bad = 0;
    for (int r = bound + blockIdx.x; r < n; r += gridDim.x) {
        const int x = perm[r];
        const int nb = nrow[r], d = nrow[r + 1] - nb;
        const int ob = d > 0 ? rowptr[x] : 0;
        const int2 vr = vrange ? vrange[x] : make_int2(0, n);
        for (int c = threadIdx.x; c < NCLASS; c += RLC_THREADS) H[c] = 0;
        __syncthreads();
        long long s1 = 0, p6 = 0, below = 0;
        for (int i = threadIdx.x; i < d; i += RLC_THREADS) {
            const int y = colidx[ob + i];
            int ys = global_id(y, vr, n);
            if (ys < 0) { bad |= ST_EINVAL; ys = x; }
            else if (ys == x || (i > 0 && y <= colidx[ob + i - 1])) bad |= ST_ENOTSIMPLE;
            const int2 vi = vinfo[ys];
            atomicAdd(&H[deg_class(vi.y)], 1);
            s1 += vi.y;
            p6 += c2m1(vi.y);
            below += vi.x < r;
        }
        s1 = warp_sum(s1);
        p6 = warp_sum(p6);
        below = warp_sum(below);
        if (lane == 0) { red[0][w] = s1; red[1][w] = p6; red[2][w] = below; }
        __syncthreads();
        if (w == 0) {
            int a0 = H[4 * lane], a1 = H[4 * lane + 1], a2 = H[4 * lane + 2], a3 = H[4 * lane + 3];
            int sum = a0 + a1 + a2 + a3;
            int ex = warp_inclusive_scan(sum) - sum;
            H[4 * lane] = ex;
            H[4 * lane + 1] = ex + a0;
            H[4 * lane + 2] = ex + a0 + a1;
            H[4 * lane + 3] = ex + a0 + a1 + a2;
        }
        __syncthreads();
        for (int k = 0; k < d; k += RLC_THREADS) {
            for (int i = threadIdx.x; i < NW * NCLASS; i += RLC_THREADS) (&wc[0][0])[i] = 0;
            __syncthreads();
            const int i = k + threadIdx.x;
            const bool act = i < d;
            int ys = act ? global_id(colidx[ob + i], vr, n) : 0;
            if (ys < 0) ys = x;
            const int2 vi = act ? vinfo[ys] : make_int2(0, 0);
            const int c = act ? deg_class(vi.y) : NCLASS + lane;
            const unsigned peers = __match_any_sync(FULL, c);
            const int rank = __popc(peers & lanemask_lt());
            if (act && rank == 0) wc[w][c] = __popc(peers);
            __syncthreads();
            if (threadIdx.x < NCLASS) {
                int s = 0;
                for (int ww = 0; ww < NW; ++ww) {
                    int t = wc[ww][threadIdx.x];
                    wc[ww][threadIdx.x] = s;
                    s += t;
                }
                tot[threadIdx.x] = s;
            }
            __syncthreads();
            if (act) ncol[nb + H[c] + wc[w][c] + rank] = vi.x;
            __syncthreads();
            if (threadIdx.x < NCLASS) H[threadIdx.x] += tot[threadIdx.x];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            long long a = 0, b = 0, c = 0;
            for (int ww = 0; ww < NW; ++ww) { a += red[0][ww]; b += red[1][ww]; c += red[2][ww]; }
            const int sp = nb + (int)c;
            rinfo[r] = make_int4(nb, sp, nb + d, 0);
            VAcc v;
            v.S1 = a; v.A1 = 0; v.P6 = b; v.A2 = 0; v.A3 = 0; v.D12 = 0; v.K4 = 0; v.C4 = 0;
            vacc[r] = v;
            red[0][0] = sp;
        }
        __syncthreads();
        const int sp = (int)red[0][0];
        for (int p = sp + threadIdx.x; p < nb + d; p += RLC_THREADS) tcnt[p] = 0;
        __syncthreads();
    }
    if (bad) set_status(status, bad);
}

static void relabel_common(const int *rowptr, const int *colidx, const int2 *vrange, Work &w, cudaStream_t st) {
    const int nt = w.ntiles;
    if (nt == 1) {   // one tile: the class order in one launch
        launch_pdl(k_class_small, 1, RS_THREADS, 0, st, rowptr, w.n, w.m, w.vinfo, w.coff, w.perm, w.nrow, w.counters,
                   w.status);
        after_launch(st, K_CLASS_HIST);
    } else {
        launch_pdl(k_class_hist, nt, RL_THREADS, 0, st, rowptr, w.n, w.m, w.vinfo, w.chist, nt, w.counters, w.status);
        after_launch(st, K_CLASS_HIST);
        launch_exclusive_scan(w.chist, w.coff, (long long)NCLASS * nt, false, w.scan_part, st);
        // ndeg (degree of each new id) is staged in `split`, then scanned into nrow
        launch_pdl(k_class_scatter, nt, RL_THREADS, 0, st, w.n, w.vinfo, w.coff, nt, w.perm, w.split);
        after_launch(st, K_CLASS_SCATTER);
        launch_exclusive_scan(w.split, w.nrow, w.n, true, w.scan_part, st);
    }
    const int lrc = w.tune[TUNE_LONG_ROW_CLASS];
    // more CTAs than an SM holds: with rows of uneven length, the later
    // waves act as load balancing
    launch_pdl(k_relabel_rows_warp, w.num_sms * w.tune[TUNE_GRID_RELABEL], 256, 0, st,
        rowptr, colidx, w.n, vrange, w.vinfo, w.perm, w.nrow, w.coff, nt, w.ncol, w.rinfo, w.vacc, w.tcnt, w.status,
        lrc);
    after_launch(st, K_RELABEL_WARP);
    launch_pdl(k_relabel_rows_cta, w.num_sms * 2, RLC_THREADS, 0, st, rowptr, colidx, w.n, vrange, w.vinfo, w.perm, w.nrow,
                                                              w.coff, nt, w.ncol, w.rinfo, w.vacc, w.tcnt,
                                                              w.status, lrc);
    after_launch(st, K_RELABEL_CTA);
}

void launch_relabel(const int *rowptr, const int *colidx, Work &w, cudaStream_t st) {
    relabel_common(rowptr, colidx, nullptr, w, st);
}

void launch_relabel_batch(const int *rowptr, const int *colidx, const int2 *vrange, Work &w, cudaStream_t st) {
    relabel_common(rowptr, colidx, vrange, w, st);
}

// Batch set-up: the union-id range of the graph that owns every vertex, and
// consistency of the offsets with rowptr.
__global__ void k_batch_setup(const int *rowptr, const long long *vo, const long long *eo, int G, int total_n,
                              int2 *vrange, int *status) {
    pdl_begin();
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (long long g = tid; g <= G; g += nthreads) {
        const long long a = vo[g];
        if (a < 0 || a > total_n || (g == 0 && a != 0) || (g == G && a != total_n)) bad = 1;
        else if (g < G && vo[g + 1] < a) bad = 1;
        else if (eo[g] != (long long)rowptr[a]) bad = 1;
    }
    for (long long x = tid; x < total_n; x += nthreads) {
        int lo = 0, hi = G - 1;  // last g with vo[g] <= x
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (vo[mid] <= x) lo = mid; else hi = mid - 1;
        }
        long long a = vo[lo], b = vo[lo + 1];
        if (a < 0 || b > total_n || a > x || b <= x) { bad = 1; a = x; b = x + 1; }
        vrange[x] = make_int2((int)a, (int)b);
    }
    if (bad) set_status(status, ST_EINVAL);
}

void launch_batch_setup(const int *rowptr, const long long *vtx_offset, const long long *edge_offset, int num_graphs,
                        int total_n, int2 *vrange, int *status, int num_sms, cudaStream_t st) {
    launch_pdl(k_batch_setup, num_sms * 4, 256, 0, st, rowptr, vtx_offset, edge_offset, num_graphs, total_n, vrange, status);
    after_launch(st, K_BATCH_SETUP);
}

}  // namespace niorca
