// niorca_api.cu -- the C ABI (include/niorca.h): argument checks, per-device
// state, work memory and the launch sequence of the three stages.
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/niorca.h"
#include "kernels.h"

namespace niorca {

void configure_stage1();
void configure_stage2();
void configure_cycle4();
void launch_batch_setup(const int *rowptr, const long long *vtx_offset, const long long *edge_offset, int num_graphs,
                        int total_n, int2 *vrange, int *status, int num_sms, cudaStream_t st);
void launch_relabel_batch(const int *rowptr, const int *colidx, const int2 *vrange, Work &w, cudaStream_t st);

// ------------------------------------------------ launch counting and timing

namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_prof_on{0};
struct Timeline {
    cudaEvent_t start = nullptr;
    std::vector<std::pair<cudaEvent_t, int>> marks;  // event after each kernel
};
std::mutex g_prof_mu;
std::vector<Timeline> g_pending;
double g_ms[K_COUNT];
long long g_calls[K_COUNT];
thread_local Timeline *t_cur = nullptr;

const char *const kNames[K_COUNT] = {
    "k_class_hist", "k_scan", "k_class_scatter", "k_relabel_rows_warp", "k_relabel_rows_cta", "k_batch_setup",
    "k_tri_warp", "k_tri_cta", "k_agg_warp", "k_agg_cta", "k_c4_warp", "k_c4_cta", "k_c4_tiled_plan",
    "k_c4_tiled", "k_solve", "k_validate", "k_c4_mid", "k_tri_big", "k_agg_big",
    "k_c4_warp_big", "k_c4_wedge_len"};
}  // namespace

const char *kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? kNames[id] : "?"; }

int resident_ctas(const void *kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n > 0 ? n : 1;
}

void after_launch(cudaStream_t st, int id) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (t_cur) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) == cudaSuccess) {
            cudaEventRecord(e, st);
            t_cur->marks.emplace_back(e, id);
        }
    }
}

namespace {

// Starts the event timeline of one call (when timing is on).
void timeline_begin(cudaStream_t st) {
    if (!g_prof_on.load()) return;
    t_cur = new Timeline();
    if (cudaEventCreate(&t_cur->start) == cudaSuccess) cudaEventRecord(t_cur->start, st);
}

void timeline_end() {
    if (!t_cur) return;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_pending.push_back(std::move(*t_cur));
    }
    delete t_cur;
    t_cur = nullptr;
}

// Waits for every recorded timeline and folds it into the totals.
void timeline_collect() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (Timeline &t : g_pending) {
        cudaEvent_t prev = t.start;
        for (auto &mk : t.marks) {
            float ms = 0.f;
            if (prev && cudaEventSynchronize(mk.first) == cudaSuccess && cudaEventElapsedTime(&ms, prev, mk.first) == cudaSuccess) {
                g_ms[mk.second] += ms;
                g_calls[mk.second] += 1;
            }
            prev = mk.first;
        }
        if (t.start) cudaEventDestroy(t.start);
        for (auto &mk : t.marks) cudaEventDestroy(mk.first);
    }
    g_pending.clear();
}

// Status words: one device int per stream that has called into the library
// on this device, so that a call reports only into the word of the stream it
// was enqueued on. The words come from one slab allocated with the device
// state (no allocation later, e.g. inside stream capture); once every word
// of the slab is taken, further streams share words by a hash of the handle.
constexpr int STATUS_WORDS = 4096;

struct DeviceState {
    bool ready = false;
    cudaMemPool_t pool = nullptr;
    int *status_slab = nullptr;
    int status_used = 0;
    std::unordered_map<const void *, int> status_of;   // stream -> word index
    int num_sms = 0;
    int tune[TUNE_COUNT] = {16, 8, 8, 8, 8, 32, 1536, 64, 1152, 8192, 12288};
};

constexpr int MAX_DEVICES = 64;
DeviceState g_dev[MAX_DEVICES];
std::mutex g_mu;

niorca_status device_state(DeviceState **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return NIORCA_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NIORCA_ECUDA;
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&d.pool, &props) != cudaSuccess) return NIORCA_ECUDA;
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (cudaMalloc(&d.status_slab, sizeof(int) * STATUS_WORDS) != cudaSuccess) return NIORCA_ENOMEM;
        if (cudaMemset(d.status_slab, 0, sizeof(int) * STATUS_WORDS) != cudaSuccess) return NIORCA_ECUDA;
        if (cudaDeviceSynchronize() != cudaSuccess) return NIORCA_ECUDA;
        configure_stage1();
        configure_stage2();
        configure_cycle4();
        if (cudaGetLastError() != cudaSuccess) return NIORCA_ECUDA;
        d.ready = true;
    }
    *out = &d;
    return NIORCA_OK;
}

// The status word of `st` on this device (see STATUS_WORDS).
int *status_word(DeviceState *ds, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_mu);
    const void *key = static_cast<const void *>(st);
    auto it = ds->status_of.find(key);
    if (it != ds->status_of.end()) return ds->status_slab + it->second;
    if (ds->status_used < STATUS_WORDS) {
        const int idx = ds->status_used++;
        ds->status_of.emplace(key, idx);
        return ds->status_slab + idx;
    }
    const uint64_t h = reinterpret_cast<uintptr_t>(key) * 0x9E3779B97F4A7C15ull;
    return ds->status_slab + (h >> 40) % STATUS_WORDS;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t vinfo, perm, chist, coff, nrow, split, rinfo, ncol, tcnt, vacc, scan_part, lists, counters, vrange;
    size_t total;
    int ntiles;
};

Layout plan(long long n, long long m, int num_sms, bool batch) {
    Layout L;
    L.ntiles = (int)((n + RL_TILE - 1) / RL_TILE);
    const long long nt = L.ntiles;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + (bytes ? bytes : 1)); return at; };
    L.vinfo = take(8 * n);
    L.perm = take(4 * n);
    L.chist = take(4 * NCLASS * nt);
    L.coff = take(4 * NCLASS * nt);
    L.nrow = take(4 * (n + 1));
    L.split = take(4 * n);
    L.rinfo = take(16 * n);
    L.ncol = take(4 * m);
    L.tcnt = take(8 * m);   // 4 m for the per-edge triangle counts; 8 m for the cursors of the 4-cycle tiles
    L.vacc = take(sizeof(VAcc) * n);
    const size_t sp1 = scan_partials(NCLASS * nt), sp2 = scan_partials(n);
    L.scan_part = take(4 * (sp1 > sp2 ? sp1 : sp2));
    L.lists = take(4 * 6 * n);
    L.counters = take(4 * NCOUNTERS);
    L.vrange = batch ? take(8 * n) : 0;
    L.total = o;
    return L;
}

niorca_status check_launch() {
    return cudaPeekAtLastError() == cudaSuccess ? NIORCA_OK : NIORCA_ECUDA;
}

// Runs the whole pipeline on one (possibly union) graph.
niorca_status run(const int *rowptr, const int *colidx, int n, int m, long long *out, cudaStream_t st,
                  const long long *vtx_offset, const long long *edge_offset, int num_graphs, int induced = 0) {
    DeviceState *ds = nullptr;
    niorca_status s = device_state(&ds);
    if (s != NIORCA_OK) return s;
    const bool batch = vtx_offset != nullptr;
    const Layout L = plan(n, m, ds->num_sms, batch);
    void *base = nullptr;
    // Inside stream capture the work memory becomes a graph allocation node
    // (plain stream-ordered allocation); otherwise it comes from the pool.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return NIORCA_ECUDA;
    const cudaError_t ae = cap == cudaStreamCaptureStatusActive ? cudaMallocAsync(&base, L.total, st)
                                                                 : cudaMallocFromPoolAsync(&base, L.total, ds->pool, st);
    if (ae != cudaSuccess) {
        cudaGetLastError();
        return NIORCA_ENOMEM;
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    Work w;
    w.n = n;
    w.m = m;
    w.ntiles = L.ntiles;
    w.vinfo = reinterpret_cast<int2 *>(b + L.vinfo);
    w.perm = reinterpret_cast<int *>(b + L.perm);
    w.chist = reinterpret_cast<int *>(b + L.chist);
    w.coff = reinterpret_cast<int *>(b + L.coff);
    w.nrow = reinterpret_cast<int *>(b + L.nrow);
    w.split = reinterpret_cast<int *>(b + L.split);
    w.rinfo = reinterpret_cast<int4 *>(b + L.rinfo);
    w.ncol = reinterpret_cast<int *>(b + L.ncol);
    w.tcnt = reinterpret_cast<int *>(b + L.tcnt);
    w.vacc = reinterpret_cast<VAcc *>(b + L.vacc);
    w.scan_part = reinterpret_cast<int *>(b + L.scan_part);
    w.lists = reinterpret_cast<int *>(b + L.lists);
    w.counters = reinterpret_cast<int *>(b + L.counters);
    w.status = status_word(ds, st);
    w.num_sms = ds->num_sms;
    for (int i = 0; i < TUNE_COUNT; ++i) w.tune[i] = ds->tune[i];
    w.induced = induced;
    cudaMemsetAsync(w.counters, 0, 4 * NCOUNTERS, st);
    timeline_begin(st);
    if (batch) {
        int2 *vrange = reinterpret_cast<int2 *>(b + L.vrange);
        launch_batch_setup(rowptr, vtx_offset, edge_offset, num_graphs, n, vrange, w.status, ds->num_sms, st);
        launch_relabel_batch(rowptr, colidx, vrange, w, st);
    } else {
        launch_relabel(rowptr, colidx, w, st);
    }
    launch_stage1(w, st);
    launch_stage2(w, st);
    launch_cycle4(w, st);
    launch_solve(w, out, st);
    timeline_end();
    s = check_launch();
    cudaFreeAsync(base, st);
    return s;
}

}  // namespace
}  // namespace niorca

using namespace niorca;

extern "C" niorca_status niorca_count(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                      int64_t *out, void *stream) {
    if (n < 0 || m < 0 || m > INT32_MAX) return NIORCA_EINVAL;
    if (n == 0) return m == 0 ? NIORCA_OK : NIORCA_EINVAL;
    if (!rowptr || !out || (m > 0 && !colidx)) return NIORCA_EINVAL;
    return run(rowptr, colidx, n, (int)m, reinterpret_cast<long long *>(out), static_cast<cudaStream_t>(stream),
               nullptr, nullptr, 0);
}

namespace {
// Whether the current device can load and store at `p` for `bytes` bytes
// from kernels: page-locked host memory (or managed/device memory), or any
// host memory where the device accesses pageable memory coherently.
bool device_reachable(const void *p, size_t bytes) {
    if (bytes == 0) return true;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return true;
    int dev = 0, pageable = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) return false;
    return pageable != 0;
}
}  // namespace

extern "C" niorca_status niorca_count_host(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                           int64_t *out, void *stream) {
    if (n < 0 || m < 0 || m > INT32_MAX) return NIORCA_EINVAL;
    if (n == 0) return m == 0 ? NIORCA_OK : NIORCA_EINVAL;
    if (!rowptr || !out || (m > 0 && !colidx)) return NIORCA_EINVAL;
    if (!device_reachable(rowptr, 4 * ((size_t)n + 1)) || !device_reachable(colidx, 4 * (size_t)m) ||
        !device_reachable(out, 120 * (size_t)n))
        return NIORCA_EINVAL;
    return run(rowptr, colidx, n, (int)m, reinterpret_cast<long long *>(out), static_cast<cudaStream_t>(stream),
               nullptr, nullptr, 0);
}

extern "C" niorca_status niorca_count_induced(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                              int64_t *out, void *stream) {
    if (n < 0 || m < 0 || m > INT32_MAX) return NIORCA_EINVAL;
    if (n == 0) return m == 0 ? NIORCA_OK : NIORCA_EINVAL;
    if (!rowptr || !out || (m > 0 && !colidx)) return NIORCA_EINVAL;
    return run(rowptr, colidx, n, (int)m, reinterpret_cast<long long *>(out), static_cast<cudaStream_t>(stream),
               nullptr, nullptr, 0, 1);
}

extern "C" niorca_status niorca_count_batch(const int32_t *rowptr, const int32_t *colidx, const int64_t *vtx_offset,
                                            const int64_t *edge_offset, int32_t num_graphs, int64_t total_n,
                                            int64_t total_m, int64_t *out, void *stream) {
    if (num_graphs < 0 || total_n < 0 || total_m < 0 || total_n > INT32_MAX - 1 || total_m > INT32_MAX)
        return NIORCA_EINVAL;
    if (num_graphs == 0 || total_n == 0) return total_m == 0 ? NIORCA_OK : NIORCA_EINVAL;
    if (!rowptr || !out || !vtx_offset || !edge_offset || (total_m > 0 && !colidx)) return NIORCA_EINVAL;
    return run(rowptr, colidx, (int)total_n, (int)total_m, reinterpret_cast<long long *>(out),
               static_cast<cudaStream_t>(stream), reinterpret_cast<const long long *>(vtx_offset),
               reinterpret_cast<const long long *>(edge_offset), num_graphs);
}

extern "C" niorca_status niorca_validate(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                         void *stream) {
    if (n < 0 || m < 0 || m > INT32_MAX) return NIORCA_EINVAL;
    if (n == 0) return m == 0 ? NIORCA_OK : NIORCA_EINVAL;
    if (!rowptr || (m > 0 && !colidx)) return NIORCA_EINVAL;
    DeviceState *ds = nullptr;
    niorca_status s = device_state(&ds);
    if (s != NIORCA_OK) return s;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    launch_validate(rowptr, colidx, n, (int)m, status_word(ds, st), ds->num_sms, st);
    return check_launch();
}

extern "C" niorca_status niorca_last_status(void *stream) {
    DeviceState *ds = nullptr;
    niorca_status s = device_state(&ds);
    if (s != NIORCA_OK) return s;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *word = status_word(ds, st);
    int bits = 0;
    // read and clear in the stream's own order, then wait for both
    if (cudaMemcpyAsync(&bits, word, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return NIORCA_ECUDA;
    if (cudaMemsetAsync(word, 0, sizeof(int), st) != cudaSuccess) return NIORCA_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return NIORCA_ECUDA;
    const niorca_status order[] = {NIORCA_EINVAL, NIORCA_ENOTSIMPLE, NIORCA_EOVERFLOW, NIORCA_ETIMEOUT};
    for (niorca_status c : order)
        if (bits & (1 << c)) return c;
    return NIORCA_OK;
}

extern "C" size_t niorca_workspace_bytes(int32_t n, int64_t m) {
    if (n <= 0 || m < 0) return 0;
    int sms = 152;
    DeviceState *ds = nullptr;
    if (device_state(&ds) == NIORCA_OK) sms = ds->num_sms;
    return plan(n, m, sms, false).total;
}

extern "C" size_t niorca_batch_workspace_bytes(int32_t num_graphs, int64_t total_n, int64_t total_m) {
    if (num_graphs <= 0 || total_n <= 0 || total_m < 0) return 0;
    int sms = 152;
    DeviceState *ds = nullptr;
    if (device_state(&ds) == NIORCA_OK) sms = ds->num_sms;
    return plan(total_n, total_m, sms, true).total;
}

extern "C" const char *niorca_status_string(niorca_status s) {
    switch (s) {
    case NIORCA_OK: return "ok";
    case NIORCA_EINVAL: return "invalid argument or CSR offsets";
    case NIORCA_ENOTSIMPLE: return "graph is not simple (self-loop, unsorted or duplicate row, asymmetric)";
    case NIORCA_EOVERFLOW: return "degree above 2^20: counts may overflow int64";
    case NIORCA_ENOMEM: return "out of device memory";
    case NIORCA_ECUDA: return "CUDA error";
    case NIORCA_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

extern "C" int32_t niorca_version(void) { return 100; }

extern "C" void niorca_profile_enable(int32_t on) { g_prof_on.store(on ? 1 : 0); }

extern "C" int32_t niorca_profile_read(double *ms, int64_t *launches, int32_t max_kernels) {
    timeline_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int i = 0; i < K_COUNT && i < max_kernels; ++i) {
        if (ms) ms[i] = g_ms[i];
        if (launches) launches[i] = g_calls[i];
    }
    return K_COUNT;
}

extern "C" void niorca_profile_reset(void) {
    timeline_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int i = 0; i < K_COUNT; ++i) { g_ms[i] = 0; g_calls[i] = 0; }
}

extern "C" const char *niorca_kernel_name(int32_t id) { return kernel_name(id); }

extern "C" int64_t niorca_launch_count(void) { return g_launches.load(); }

namespace {
bool tune_valid(int i, int v) {
    switch (i) {
    case TUNE_LONG_ROW_CLASS: return v >= 1 && v < NCLASS;
    case TUNE_C4_WARP_MAXW: return v >= 2 && v <= 1536;
    case TUNE_WARP_MAXD: return v >= 2 && v <= 64;
    case TUNE_TRI_BITS_MAXD: return v >= 2 && v <= 1152;
    case TUNE_TRI_HASH_MAXD: return v >= 2 && v <= 8192;
    case TUNE_C4_TEAM_MINW: return v >= 2 && v <= 12288;
    default: return v >= 1 && v <= 64;   // CTAs per SM
    }
}
}  // namespace

extern "C" niorca_status niorca_set_tuning(const int32_t *values, int32_t count) {
    if (!values || count < 0 || count > TUNE_COUNT) return NIORCA_EINVAL;
    for (int i = 0; i < count; ++i)
        if (!tune_valid(i, values[i])) return NIORCA_EINVAL;
    DeviceState *ds = nullptr;
    niorca_status s = device_state(&ds);
    if (s != NIORCA_OK) return s;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < count; ++i) ds->tune[i] = values[i];
    return NIORCA_OK;
}

extern "C" int32_t niorca_get_tuning(int32_t *values, int32_t count) {
    DeviceState *ds = nullptr;
    if (device_state(&ds) != NIORCA_OK) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < count && i < TUNE_COUNT; ++i) values[i] = ds->tune[i];
    return TUNE_COUNT;
}
