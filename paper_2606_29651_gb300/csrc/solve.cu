// solve.cu -- Stage III-b: the orbit equations (Sec. 5 and the Appendix).
//
// For every vertex x the neighbours' S1 (sum of their neighbours' degrees)
// and A1 (twice their triangle count) are summed over N(x); together with
// x's own accumulators this gives the nine f* variables of Table 1 in closed
// form (each is a sum over the substructures of Fig. 3 around x):
//   f_12^14 = D12
//   f_10^13 = A3 - 2 A1 - 2 D12
//   f_13^14 = A2 - A1
//   f_11^13 = (d - 1) A1 - A2
//   f_5^8   = (d - 1)(S1 - d) - (d - 1) A1 - (A3 - A1) + A2
//   f_6^9   = 2 P6 - 2 A3 + 3 A1 + A2
//   f_9^12  = 2 sum_y T(y) - 2 A1 - 2 D12
//   f_4^8   = sum_y S1(y) - S1 - 2 sum_y T(y) - d (d - 1) + A1 - f_10^13
//   f_8^12  = 2 C4 - f_13^14
// with d = deg x, T = A1 / 2 and sum_y over N(x). The equations of the paper
// then give psi_4 .. psi_13; psi_0 = d, psi_1 = S1 - d (paths x-y-z),
// psi_2 = C(d, 2), psi_3 = T, psi_7 = C(d, 3), psi_14 = K4. Rows are written
// in the caller's vertex ids.
#include "kernels.h"

namespace niorca {

__device__ __forceinline__ void orbit_equations(long long d, const VAcc &a, long long sS1, long long sT,
                                                long long *psi) {
    const long long A1 = a.A1, A2 = a.A2, A3 = a.A3, S1 = a.S1, D12 = a.D12;
    const long long f12 = D12;
    const long long f10 = A3 - 2 * A1 - 2 * D12;
    const long long f13 = A2 - A1;
    const long long f11 = (d - 1) * A1 - A2;
    const long long f5 = (d - 1) * (S1 - d) - (d - 1) * A1 - (A3 - A1) + A2;
    const long long f6 = 2 * a.P6 - 2 * A3 + 3 * A1 + A2;
    const long long f9 = 2 * sT - 2 * A1 - 2 * D12;
    const long long f4 = sS1 - S1 - 2 * sT - d * (d - 1) + A1 - f10;
    const long long f8 = 2 * a.C4 - f13;
    psi[0] = d;
    psi[1] = S1 - d;
    psi[2] = d * (d - 1) / 2;
    psi[3] = A1 / 2;
    psi[4] = 2 * f12 + f4 + f10 + f9;          // Appendix, o4
    psi[5] = 2 * f12 + f5 + f10 + f11;         // Appendix, o5
    psi[6] = (f6 - f13) / 2 + f10 + 2 * f12;   // Appendix, o6
    psi[7] = d * (d - 1) / 2 * (d - 2) / 3;    // Appendix, o7 = C(psi_0, 3)
    psi[8] = (f13 + f8) / 2;                   // Appendix, o8
    psi[9] = f12 + f9 / 2;                     // Appendix, o9
    psi[10] = f10 + 2 * f12;                   // Eq. o10
    psi[11] = (f11 + f13) / 2;                 // Eq. o11
    psi[12] = f12;                             // Eq. o12
    psi[13] = f13 / 2;                         // Eq. o13
    psi[14] = a.K4;                            // K4[x] (Stage II)
}

// Induced counts from non-induced ones. An induced graphlet with x in
// orbit j contains a fixed number of spanning non-induced graphlets with x
// in orbit k (psi = O psi', O unitriangular; e.g. a K4 holds six paths with
// x at an end, three diamonds with x of degree 3). Back-substitution from
// the densest graphlet down; the rows for o13, o11 and o10 are the induced
// equations printed in Sec. 5 (psi'13 = f13/2 - 3 f14, psi'11 =
// (f11 - f13)/2 + 3 f14, psi'10 = f10 - f13 + 6 f14).
__device__ __forceinline__ void to_induced(long long *p) {
    const long long i14 = p[14];
    const long long i13 = p[13] - 3 * i14;
    const long long i12 = p[12] - 3 * i14;
    const long long i11 = p[11] - 2 * i13 - 3 * i14;
    const long long i10 = p[10] - 2 * i12 - 2 * i13 - 6 * i14;
    const long long i9 = p[9] - 2 * i12 - 3 * i14;
    const long long i8 = p[8] - i12 - i13 - 3 * i14;
    const long long i7 = p[7] - i11 - i13 - i14;
    const long long i6 = p[6] - i9 - i10 - 2 * i12 - i13 - 3 * i14;
    const long long i5 = p[5] - 2 * i8 - i10 - 2 * i11 - 2 * i12 - 4 * i13 - 6 * i14;
    const long long i4 = p[4] - 2 * i8 - 2 * i9 - i10 - 4 * i12 - 2 * i13 - 6 * i14;
    const long long i3 = p[3];
    p[1] -= 2 * i3;
    p[2] -= i3;
    p[4] = i4; p[5] = i5; p[6] = i6; p[7] = i7; p[8] = i8; p[9] = i9;
    p[10] = i10; p[11] = i11; p[12] = i12; p[13] = i13; p[14] = i14;
}

// Rows from the long-row class on (new ids from `bound`, the degree-class
// order puts them last): one warp per vertex. Every other vertex is solved in
// groups of 32 consecutive caller ids: each lane loads its vertex's row bounds
// and accumulators up front, the warp sums S1 and A1 over the neighbours of
// each of the 32 in turn (coalesced gathers, two vertices in flight), each
// lane solves its own vertex, and the warp writes the group's 32 output rows
// (3840 contiguous bytes) with coalesced stores through shared memory, which
// also suits an output buffer in host memory. With long_class 0 (a graph
// with fewer vertices than the grid has warps) every vertex takes a warp.
__device__ __forceinline__ void solve_write(long long d, const VAcc &a, long long sS1, long long sA1, int induced,
                                            long long *o) {
    long long psi[15];
    orbit_equations(d, a, sS1, sA1 / 2, psi);
    if (induced) to_induced(psi);
#pragma unroll
    for (int k = 0; k < 15; ++k) o[k] = psi[k];
}

constexpr int SOLVE_WARPS = 8;

__global__ void __launch_bounds__(SOLVE_WARPS * 32) k_solve(Graph g, const VAcc *vacc, const int *perm,
                                                            const int2 *vinfo, long long *out, int induced,
                                                            const int *coff, int ntiles, int long_class,
                                                            const int *counters) {
    pdl_begin();
    __shared__ long long obuf[SOLVE_WARPS][32 * 15];
    if (degree_overflow(counters)) return;
    const int lane = lane_id();
    long long *ob = obuf[threadIdx.x >> 5];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int bound = min(coff[long_class * ntiles], g.n);
    for (int x = bound + gw; x < g.n; x += nw) {
        const int4 rx = g.rinfo[x];
        long long sS1 = 0, sA1 = 0;
        for (int p = rx.x + lane; p < rx.z; p += 32) {
            const longlong2 sa = *reinterpret_cast<const longlong2 *>(&vacc[g.ncol[p]]);
            sS1 += sa.x;
            sA1 += sa.y;
        }
        sS1 = warp_sum(sS1);
        sA1 = warp_sum(sA1);
        if (lane == 0) solve_write(rx.z - rx.x, vacc[x], sS1, sA1, induced, out + (size_t)perm[x] * 15);
    }
    for (int xo0 = gw * 32; long_class > 0 && xo0 < g.n; xo0 += nw * 32) {
        const int xo = xo0 + lane;   // caller id
        int x = -1;                  // relabelled id, if this group solves it
        if (xo < g.n) {
            const int2 vi = vinfo[xo];
            if (deg_class(vi.y) < long_class) x = vi.x;
        }
        const bool have = x >= 0;
        const unsigned mine = __ballot_sync(FULL, have);
        int4 rx = make_int4(0, 0, 0, 0);
        VAcc a{};
        if (have) {
            rx = g.rinfo[x];
            a = vacc[x];
        }
        long long mS1 = 0, mA1 = 0;   // this lane's vertex
        const int cnt = min(32, g.n - xo0);
        for (int k = 0; k < cnt; k += 2) {
            const int b0 = __shfl_sync(FULL, rx.x, k), e0 = __shfl_sync(FULL, rx.z, k);
            const int b1 = __shfl_sync(FULL, rx.x, k + 1 < 32 ? k + 1 : 31);
            const int e1 = k + 1 < cnt ? __shfl_sync(FULL, rx.z, k + 1) : b1;
            long long s0 = 0, t0 = 0, s1 = 0, t1 = 0;
            for (int off = lane; off < max(e0 - b0, e1 - b1); off += 32) {
                if (b0 + off < e0) {
                    const longlong2 sa = *reinterpret_cast<const longlong2 *>(&vacc[g.ncol[b0 + off]]);
                    s0 += sa.x;
                    t0 += sa.y;
                }
                if (b1 + off < e1) {
                    const longlong2 sa = *reinterpret_cast<const longlong2 *>(&vacc[g.ncol[b1 + off]]);
                    s1 += sa.x;
                    t1 += sa.y;
                }
            }
            s0 = warp_sum(s0);
            t0 = warp_sum(t0);
            s1 = warp_sum(s1);
            t1 = warp_sum(t1);
            if (lane == k) { mS1 = s0; mA1 = t0; }
            if (lane == k + 1) { mS1 = s1; mA1 = t1; }
        }
        if (have) solve_write(rx.z - rx.x, a, mS1, mA1, induced, ob + lane * 15);
        __syncwarp();
        long long *o = out + (size_t)xo0 * 15;
        for (int i = lane; i < cnt * 15; i += 32)
            if ((mine >> (i / 15)) & 1u) o[i] = ob[i];
        __syncwarp();
    }
}

void launch_solve(Work &w, long long *out, cudaStream_t st) {
    Graph g{w.n, w.m, w.rinfo, w.ncol};
    const int grid = w.num_sms * w.tune[TUNE_GRID_SOLVE];
    // a graph with no more vertices than the grid has warps: one warp per
    // vertex (long_class 0), so that no warp solves 32 vertices in turn
    const int lc = (long long)w.n <= (long long)grid * SOLVE_WARPS ? 0 : w.tune[TUNE_LONG_ROW_CLASS];
    launch_pdl(k_solve, grid, SOLVE_WARPS * 32, 0, st,
        g, w.vacc, w.perm, w.vinfo, out, w.induced, w.coff, w.ntiles, lc, w.counters);
    after_launch(st, K_SOLVE);
}

// Full simple-graph check: offsets, strictly increasing rows, no self-loops,
// and symmetry (every (x, y) has its (y, x)), one warp per row.
__global__ void __launch_bounds__(256) k_validate(const int *rowptr, const int *colidx, int n, int m, int *status) {
    pdl_begin();
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int bad = 0;
    for (int x = gw; x < n; x += nw) {
        const int a = rowptr[x], b = rowptr[x + 1];
        if (a < 0 || b < a || b > m || (x == 0 && a != 0) || (x == n - 1 && b != m)) {
            bad |= ST_EINVAL;
            continue;
        }
        for (int p = a + lane; p < b; p += 32) {
            const int y = colidx[p];
            if (y < 0 || y >= n) { bad |= ST_EINVAL; continue; }
            if (y == x || (p > a && colidx[p - 1] >= y)) { bad |= ST_ENOTSIMPLE; continue; }
            const int ya = rowptr[y], yb = rowptr[y + 1];
            if (ya < 0 || yb < ya || yb > m) { bad |= ST_EINVAL; continue; }
            if (find_sorted(colidx, ya, yb, x) < 0) bad |= ST_ENOTSIMPLE;
        }
    }
    bad = __reduce_or_sync(FULL, bad);
    if (lane == 0 && bad) set_status(status, bad);
}

void launch_validate(const int *rowptr, const int *colidx, int n, int m, int *status, int num_sms, cudaStream_t st) {
    if (n <= 0) return;
    launch_pdl(k_validate, num_sms * 8, 256, 0, st, rowptr, colidx, n, m, status);
    after_launch(st, K_VALIDATE);
}

}  // namespace niorca
