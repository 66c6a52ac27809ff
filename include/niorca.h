/*
 * niorca.h -- C ABI of the GB300 NI-ORCA library (libniorca.so).
 *
 * The library computes, for every vertex x of a simple undirected graph
 * G = (V, E), the counts psi_0(x) .. psi_14(x) of the 15 orbits of the
 * non-induced connected graphlets on 2, 3 and 4 vertices (Sec. 3, Defs. 3-5;
 * the output o_0 .. o_14 of Algorithm 1). It follows the paper's three
 * stages: per-edge triangles (Stage I, Algorithm 1), 4-cliques (Stage II,
 * Algorithm 2) and the orbit equations over the f* variables of Table 1
 * (Stage III, Sec. 5 and the Appendix). Every count is an exact int64.
 *
 * Orbit numbering (the paper's Fig. 2 is not in its text; the numbering
 * under which all its equations hold): 0 edge; 1 / 2 end / middle of a path
 * on 3 vertices; 3 triangle; 4 / 5 end / interior of a path on 4 vertices;
 * 6 / 7 leaf / centre of a 3-star; 8 4-cycle; 9 / 10 / 11 vertex of degree
 * 1 / 2 / 3 of the paw (tailed triangle); 12 / 13 vertex of degree 2 / 3 of
 * the diamond; 14 K4.
 *
 * Conventions for every call:
 *   - Graph input is CSR in caller-owned DEVICE memory: rowptr int32[n+1]
 *     with rowptr[0] = 0 and rowptr[n] = m; colidx int32[m]; m = 2|E| (each
 *     undirected edge appears in both rows). Every row is strictly increasing,
 *     has no self-loop, and the graph is symmetric (Sec. 3: a simple graph).
 *   - Output is caller-owned DEVICE memory, int64 out[n * 15], row-major:
 *     out[v * 15 + k] = psi_k(v). It is fully overwritten.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls
 *     only enqueue work; they never synchronise the stream. Results are valid
 *     once the stream has reached the end of the call's work. The kernels are
 *     launched with programmatic dependent launch allowed: a kernel may be
 *     scheduled while the one before it on the stream drains, and waits for
 *     it to complete (griddepcontrol.wait) before it touches memory, so the
 *     stream order with the caller's own work is unchanged. No kernel of the
 *     library lets the work after it start early.
 *   - Argument errors are returned synchronously and nothing is enqueued.
 *     Errors found on the device (malformed CSR, too large a degree) are
 *     recorded in the status word of the call's stream, read by
 *     niorca_last_status(stream); after such an error `out` is unspecified.
 *     Malformed input never makes a kernel access memory outside the given
 *     arrays: a degree above 2^20 stops every stage after the degree pass.
 *   - Work memory is taken from a library-owned, stream-ordered pool on the
 *     current device and returned to it when the stream reaches the end of
 *     the call; the pool keeps freed memory for reuse.
 *   - Sizes: n < 2^31, m < 2^31; the largest degree must be at most 2^20,
 *     which bounds every intermediate below 2^62 (else NIORCA_EOVERFLOW).
 */
#ifndef NIORCA_H
#define NIORCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NIORCA_OK = 0,
    NIORCA_EINVAL = 1,      /* bad argument, or CSR offsets out of range      */
    NIORCA_ENOTSIMPLE = 2,  /* self-loop, unsorted/duplicate row, asymmetric   */
    NIORCA_EOVERFLOW = 3,   /* a degree above 2^20: counts may exceed int64    */
    NIORCA_ENOMEM = 4,      /* the work memory could not be allocated          */
    NIORCA_ECUDA = 5,       /* a CUDA call failed (launch, pool, event)        */
    NIORCA_ETIMEOUT = 6     /* a bounded device wait gave up                   */
} niorca_status;

/*
 * Orbit counts of one graph (Algorithm 1: Stages I, II and III).
 *   rowptr  device int32[n + 1]   CSR offsets, rowptr[0] = 0, rowptr[n] = m
 *   colidx  device int32[m]       neighbours, each row strictly increasing
 *   n       number of vertices, 0 <= n < 2^31
 *   m       number of CSR entries (2|E|), 0 <= m < 2^31
 *   out     device int64[n * 15]  psi_k(v) at out[v * 15 + k]
 *   stream  cudaStream_t to enqueue on
 * Returns NIORCA_EINVAL for null pointers with n > 0 or m > 0, negative or
 * too large sizes; NIORCA_ENOMEM / NIORCA_ECUDA if enqueueing failed.
 */
niorca_status niorca_count(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                           int64_t *out, void *stream);

/*
 * Orbit counts of one graph whose CSR and output live in HOST memory, with
 * no staging copy: the kernels that read the CSR (the degree-class pass and
 * the row relabelling, each reading it once in order) load it across the
 * host link, and the orbit solve stores the counts into `out` in blocks of
 * 32 contiguous rows. On GB300 (Grace host, NVLink-C2C) the transfers thus
 * overlap the kernels instead of preceding and following them.
 *   rowptr  host int32[n + 1], colidx host int32[m], out host int64[n * 15],
 *           same meaning and layout as niorca_count; each must be
 *           page-locked (cudaHostAlloc / cudaHostRegister) or reachable by
 *           the device through coherent access to pageable memory. The
 *           caller keeps them alive and unmodified until the stream reaches
 *           the end of the call; `out` is complete only then.
 *   stream  cudaStream_t to enqueue on
 * Device pointers are accepted too. Returns NIORCA_EINVAL for a buffer the
 * device cannot reach, otherwise as niorca_count. The paper has no
 * counterpart: it concerns how the input reaches the GPU, not the method.
 */
niorca_status niorca_count_host(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                int64_t *out, void *stream);

/*
 * INDUCED orbit counts psi'_k(v) of one graph: the graphlet must be the
 * subgraph induced by its vertices (Def. 2), the variant ORCA counts and
 * that Sec. 5 contrasts with NI-ORCA (psi'13, psi'11, psi'10 are printed
 * there). Computed from the non-induced counts of the same three stages;
 * arguments and errors as niorca_count.
 */
niorca_status niorca_count_induced(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                   int64_t *out, void *stream);

/*
 * Orbit counts of many independent graphs in one call (the same stages for
 * each graph; graphs are packed back to back).
 *   rowptr      device int32[total_n + 1]: the concatenation of every
 *               graph's offsets rowptr_g[0..n_g-1], each shifted by
 *               edge_offset[g], followed by total_m. Equivalently the CSR of
 *               the disjoint union of the graphs.
 *   colidx      device int32[total_m]: column ids LOCAL to each graph
 *               (0 <= colidx < n_g).
 *   vtx_offset  device int64[num_graphs + 1]: prefix sums of n_g.
 *   edge_offset device int64[num_graphs + 1]: prefix sums of m_g.
 *   num_graphs  number of graphs (>= 0).
 *   total_n, total_m  vtx_offset[num_graphs] and edge_offset[num_graphs].
 *   out         device int64[total_n * 15]; graph g's vertex v at row
 *               vtx_offset[g] + v.
 * Each graph is subject to the limits of niorca_count. The results are
 * identical to counting each graph alone.
 */
niorca_status niorca_count_batch(const int32_t *rowptr, const int32_t *colidx, const int64_t *vtx_offset,
                                 const int64_t *edge_offset, int32_t num_graphs, int64_t total_n,
                                 int64_t total_m, int64_t *out, void *stream);

/*
 * Full simple-graph check of a CSR (Sec. 3: G is simple and undirected):
 * offsets in range, rows strictly increasing, no self-loops, and every
 * entry (x, y) matched by (y, x). Enqueued on `stream`; the verdict is
 * read with niorca_last_status(). niorca_count itself checks everything
 * but symmetry.
 */
niorca_status niorca_validate(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m, void *stream);

/*
 * Reads and clears the status word of `stream` on the current device, in
 * the stream's order, and synchronises the stream: the errors that calls
 * enqueued on this stream recorded since the previous read (NIORCA_OK if
 * none; the lowest code if several), or NIORCA_ECUDA if the stream itself
 * reports an error. Calls on other streams never set or clear this word, so
 * concurrent calls on separate streams report separately. A call captured
 * into a CUDA graph reports into the word of the stream it was captured on.
 * The library holds 4096 words per device; beyond 4096 distinct streams,
 * streams share words (by a hash of the handle) and may see each other's
 * errors.
 */
niorca_status niorca_last_status(void *stream);

/*
 * Orbit counts of one graph without allocating any memory. The paper has no
 * counterpart: this exists for callers that must not allocate device memory
 * or let a library do so -- code whose device memory is owned and budgeted
 * by a host application or framework (a plugin in another program's CUDA
 * context, a runtime that hands out only its own buffers), or a system that
 * forbids allocation once it is running. The counts are those of
 * niorca_count.
 *   rowptr, colidx, n, m, out, stream  as niorca_count
 *   status  device int32 or NULL. The call sets it to 0, then ORs in bit k
 *           for every device-detected error with code k (same codes as the
 *           return value). With NULL such errors are not reported.
 * Work memory: one static device array of NIORCA_NOALLOC_SCRATCH_BYTES
 * (64 MiB) inside the library, which every GPU that loads the library holds
 * until the process exits. A graph whose work memory does not fit (roughly
 * 130 n + 8 m bytes, e.g. n = 1e5 with m = 4e6) is rejected with
 * NIORCA_ENOMEM before anything is enqueued. The call uses the default
 * launch shape, not niorca_set_tuning's.
 * The first call on a device finds the array's device address (set-up, no
 * allocation); make that first call before any stream capture. Every call
 * on a device shares the one array: calls whose work overlaps on the GPU
 * (different streams, no ordering between them) race and give wrong counts;
 * calls on one stream, or otherwise ordered, are fine. The array keeps the
 * last call's contents; each call clears what must start at zero.
 */
#define NIORCA_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
niorca_status niorca_count_noalloc(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                   int64_t *out, int32_t *status, void *stream);

/* Bytes of work memory one niorca_count call of this size takes. */
size_t niorca_workspace_bytes(int32_t n, int64_t m);

/* Work memory of a niorca_count_batch call of this size. */
size_t niorca_batch_workspace_bytes(int32_t num_graphs, int64_t total_n, int64_t total_m);

/* Human-readable name of a status code (static string). */
const char *niorca_status_string(niorca_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t niorca_version(void);

/*
 * Tracing (no counterpart in the paper, which reports PAPI counters; here
 * CUDA events). When enabled, every kernel the library launches is followed
 * by an event on the call's stream, so the time of each kernel is the gap
 * between consecutive events. Keep it off while capturing a CUDA graph.
 *   niorca_profile_enable  switch per-kernel timing on (1) or off (0).
 *   niorca_profile_read    waits for the recorded events, then writes the
 *                          accumulated milliseconds and launch counts of
 *                          every kernel id (0 .. return value - 1) into
 *                          ms[] and launches[] (either may be NULL; at most
 *                          max_kernels entries). Returns the number of ids.
 *   niorca_profile_reset   clears the totals.
 *   niorca_kernel_name     name of a kernel id (static string).
 *   niorca_launch_count    kernels launched by the library since it was
 *                          loaded, timing on or off.
 */
/*
 * Tuning of the launch shape (no counterpart in the paper, whose knobs are
 * OpenMP schedules and chunk sizes, Sec. 8). values[i] for i < count sets,
 * for the current device and every later call on it:
 *   0..4  CTAs per SM of the relabel, triangle, edge-aggregate, 4-cycle and
 *         solve kernels (1..64; defaults 16, 8, 8, 8, 8)
 *   5     degree class from which a row is relabelled by a whole CTA
 *         (1..127; default 32, i.e. degree >= 512)
 *   6     largest wedge count W of a 4-cycle root handled by one warp (2..1536)
 *   7     largest out-degree of a triangle root handled by one warp (2..64)
 *   8     largest out-degree of a CTA-tier triangle root that keeps the bit
 *         matrix of its out-neighbourhood (2..1152; default 1152)
 *   9     largest out-degree of a CTA-tier triangle root that hashes its
 *         out-neighbourhood in shared memory; above it, binary searches
 *         (2..8192; default 8192)
 *   10    4-cycle roots with more wedges than this are counted by the
 *         key-tiled tier (2..12288; default 12288)
 * Any setting gives the same counts; only the speed changes. Returns
 * NIORCA_EINVAL (and changes nothing) for a value out of range.
 * niorca_get_tuning copies the current values and returns how many exist.
 */
niorca_status niorca_set_tuning(const int32_t *values, int32_t count);
int32_t niorca_get_tuning(int32_t *values, int32_t count);

void niorca_profile_enable(int32_t on);
int32_t niorca_profile_read(double *ms, int64_t *launches, int32_t max_kernels);
void niorca_profile_reset(void);
const char *niorca_kernel_name(int32_t id);
int64_t niorca_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* NIORCA_H */
