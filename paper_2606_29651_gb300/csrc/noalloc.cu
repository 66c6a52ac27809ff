// noalloc.cu -- orbit counting that allocates no memory.
//
// niorca_count takes its work memory from a pool that the library grows
// with stream-ordered allocation. Some callers cannot allow that: code that
// runs inside a host application whose device memory is owned and budgeted
// by someone else (a framework that only hands out its own tensors, a plugin
// living in another program's CUDA context), or a runtime that forbids any
// allocation after start-up. niorca_count_noalloc serves them: the caller
// passes the graph and the output as usual, and every byte of work memory
// comes from one array compiled into this file. The array is a file-scope
// static __device__ object, so every GPU that loads the library holds it
// (NIORCA_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// In host code the array's name only stands in for the device object; its
// device address is obtained once per device with cudaGetSymbolAddress and
// passed to the kernels. The kernels are the same as niorca_count's.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/niorca.h"
#include "kernels.h"

namespace niorca {

void configure_stage1();
void configure_stage2();
void configure_cycle4();

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NIORCA_NOALLOC_SCRATCH_BYTES];
static __device__ int g_noalloc_status;   // error bits when the caller passes no status word

struct NoallocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    int *status = nullptr;              // device address of g_noalloc_status
    int num_sms = 0;
};

constexpr int kMaxDevices = 64;
NoallocDevice g_na[kMaxDevices];
std::mutex g_na_mu;

// First call on a device: find the device addresses of the static objects.
niorca_status noalloc_setup(NoallocDevice **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NIORCA_ECUDA;
    std::lock_guard<std::mutex> lk(g_na_mu);
    NoallocDevice &d = g_na[dev];
    if (!d.ready) {
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&d.scratch), g_noalloc_scratch) != cudaSuccess)
            return NIORCA_ECUDA;
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&d.status), g_noalloc_status) != cudaSuccess)
            return NIORCA_ECUDA;
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return NIORCA_ECUDA;
        configure_stage1();
        configure_stage2();
        configure_cycle4();
        if (cudaGetLastError() != cudaSuccess) return NIORCA_ECUDA;
        d.ready = true;
    }
    *out = &d;
    return NIORCA_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves the static array into the buffers of one call; returns the bytes
// needed (which may exceed the array; the caller checks).
size_t carve(unsigned char *base, long long n, long long m, Work *w) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + o;
        o = up256(o + (bytes ? bytes : 1));
        return p;
    };
    const long long nt = (n + RL_TILE - 1) / RL_TILE;
    w->vinfo = reinterpret_cast<int2 *>(take(8 * n));
    w->perm = reinterpret_cast<int *>(take(4 * n));
    w->chist = reinterpret_cast<int *>(take(4 * NCLASS * nt));
    w->coff = reinterpret_cast<int *>(take(4 * NCLASS * nt));
    w->nrow = reinterpret_cast<int *>(take(4 * (n + 1)));
    w->split = reinterpret_cast<int *>(take(4 * n));
    w->rinfo = reinterpret_cast<int4 *>(take(16 * n));
    w->ncol = reinterpret_cast<int *>(take(4 * m));
    w->tcnt = reinterpret_cast<int *>(take(8 * m));   // also the cursors of the key-tiled 4-cycle tier
    w->vacc = reinterpret_cast<VAcc *>(take(sizeof(VAcc) * n));
    const size_t sp1 = scan_partials(NCLASS * nt), sp2 = scan_partials(n);
    w->scan_part = reinterpret_cast<int *>(take(4 * (sp1 > sp2 ? sp1 : sp2)));
    w->lists = reinterpret_cast<int *>(take(4 * 6 * n));
    w->counters = reinterpret_cast<int *>(take(4 * NCOUNTERS));
    w->ntiles = (int)nt;
    return o;
}

}  // namespace
}  // namespace niorca

using namespace niorca;

extern "C" niorca_status niorca_count_noalloc(const int32_t *rowptr, const int32_t *colidx, int32_t n, int64_t m,
                                              int64_t *out, int32_t *status, void *stream) {
    if (n < 0 || m < 0 || m > INT32_MAX) return NIORCA_EINVAL;
    if (n == 0) return m == 0 ? NIORCA_OK : NIORCA_EINVAL;
    if (!rowptr || !out || (m > 0 && !colidx)) return NIORCA_EINVAL;
    NoallocDevice *d = nullptr;
    niorca_status s = noalloc_setup(&d);
    if (s != NIORCA_OK) return s;
    Work w;
    const size_t need = carve(d->scratch, n, m, &w);
    if (need > NIORCA_NOALLOC_SCRATCH_BYTES) return NIORCA_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    w.n = n;
    w.m = (int)m;
    w.status = status ? reinterpret_cast<int *>(status) : d->status;
    w.num_sms = d->num_sms;
    if (cudaMemsetAsync(w.status, 0, sizeof(int), st) != cudaSuccess) return NIORCA_ECUDA;
    if (cudaMemsetAsync(w.counters, 0, 4 * NCOUNTERS, st) != cudaSuccess) return NIORCA_ECUDA;
    launch_relabel(rowptr, colidx, w, st);
    launch_stage1(w, st);
    launch_stage2(w, st);
    launch_cycle4(w, st);
    launch_solve(w, reinterpret_cast<long long *>(out), st);
    return cudaPeekAtLastError() == cudaSuccess ? NIORCA_OK : NIORCA_ECUDA;
}
