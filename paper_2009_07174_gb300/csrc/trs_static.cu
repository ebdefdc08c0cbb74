// trs_static.cu -- trs_normalize_static: normalise one term without any
// memory allocation, for callers that cannot allocate device memory (a
// real-time or embedded host loop that forbids allocator calls after start-up,
// code running while the caller's memory pool is locked, or a process whose
// device memory is fully reserved by another framework).  The node store lives
// in a file-scope device array of fixed size; the caller passes the input term
// and the output buffer as device pointers.
//
// Limits and sharing: the array holds kStaticBytes bytes on every GPU that
// loads the library, until the process exits.  Every call uses the same array
// and leaves its contents behind; the call clears the control block and the
// slots it uses before starting.  Two calls whose GPU work overlaps (different
// streams, or different host threads) race on the array and corrupt each
// other's results: serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>

#include "trs_engine.h"

namespace trs {
size_t engine_smem_bytes(const DevPool &P, int mode, int block);
cudaError_t engine_configure(int mode, int block, size_t smem, int *blocks_per_sm, const void *fn = nullptr);
cudaError_t engine_launch(const DevPool &P, const LaunchOpts &o, long long budget,
                          unsigned long long cond, cudaStream_t stream, const void *fn = nullptr);
cudaError_t prep_launch(Ctl *ctl, long long max_sweeps, int seed, cudaStream_t stream);

namespace {

constexpr size_t kStaticBytes = 24u << 20;  // 24 MiB per GPU
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mu;
unsigned char *g_addr[kMaxDevices];  // device address of the array, per device

size_t up(size_t x) { return (x + 255) / 256 * 256; }

// Carve the array: control block, trace, rule table, then the per-slot arrays.
// Returns the number of slots that fit (0 if the table alone does not fit).
long long carve(unsigned char *base, const Program &p, DevPool *d)
{
    size_t off = 0;
    d->ctl = (Ctl *)(base + off);
    off = up(off + sizeof(Ctl));
    d->trace = (trs_sweep_record *)(base + off);
    d->trace_cap = 1;
    off = up(off + sizeof(trs_sweep_record));
    d->tab = (const int32_t *)(base + off);
    d->tab_words = (int32_t)p.table.size();
    off = up(off + p.table.size() * sizeof(int32_t));
    const int rs = rec_stride(p.maxarity);
    // record, nfs, ring, fq0, fq1 (the frontier buffers double as stacks), the
    // collection's candidate list; and one bit per slot (candidate bitmap)
    const int words = rs + 6;
    if (off + (size_t)7 * 256 >= kStaticBytes) return 0;
    long long cap = (long long)((kStaticBytes - off - (size_t)7 * 256) * 8 / ((size_t)words * 32 + 1));
    cap = cap / 64 * 64;
    auto take = [&](size_t n) { unsigned char *at = base + off; off = up(off + n); return (int32_t *)at; };
    const size_t s = (size_t)cap * 4;
    d->rec = take(s * rs);
    d->rs = rs;
    d->nfs = take(s);
    d->ring = take(s);
    d->fq[0] = take(s);
    d->fq[1] = take(s);
    d->cand = take(s);
    d->dbm = (uint32_t *)take((size_t)(cap + 31) / 32 * 4);
    d->act = nullptr;
    d->cap = cap;
    d->ma = p.maxarity;
    return cap;
}

// Build the tree of the preorder term d_term in slots 1 .. len (one thread:
// the sizes this entry point accepts are small).  Clears the slot arrays it
// uses and slot 0.
__global__ void k_static_upload(DevPool P, const int32_t *term, long long len, int32_t *stk_node,
                                int32_t *stk_next)
{
    Ctl *c = P.ctl;
    const int32_t *ar = P.tab + P.tab[4];  // arity in the low byte of each word
    const int32_t nsym = P.tab[1];
    for (int w = 0; w < P.rs; w++) P.rec[w] = 0;
    P.nfs[0] = 0;
    long long sp = 0;
    for (long long q = 0; q < len; q++) {
        const int32_t s = term[q];
        if (s <= 0 || s >= nsym || (q > 0 && sp == 0)) { c->status = TRS_ERR_BAD_TERM; return; }
        const int32_t node = (int32_t)(q + 1);
        for (int w = 0; w < P.rs; w++) node_at(P, node)[w] = 0;
        hs_at(P, node) = s;
        rc_at(P, node) = 1;
        P.nfs[node] = -1;
        if (sp > 0) {
            int32_t parent = stk_node[sp - 1];
            int32_t j = stk_next[sp - 1]++;
            arg_at(P, j, parent) = node;
            // the parent word: sign bit set when the parent's head is unary
            par_at(P, node) = parent | ((ar[hs_at(P, parent)] & 0xff) == 1 ? (int32_t)0x80000000 : 0);
            if (stk_next[sp - 1] == (ar[hs_at(P, parent)] & 0xff)) sp--;
        }
        if ((ar[s] & 0xff) > 0) { stk_node[sp] = node; stk_next[sp] = 0; sp++; }
    }
    if (sp != 0) { c->status = TRS_ERR_BAD_TERM; return; }
    c->sweep_id = 1;
    c->n_top = len + 1;
    c->fl_begin = c->fl_end = 0;
    c->dead = 0;
}

// Preorder of the tree at slot 1 into out[0 .. out_cap); *out_len receives
// its length, or -1 with TRS_ERR_BUFFER_SMALL in the status if it does not fit.
__global__ void k_static_download(DevPool P, int32_t *out, long long out_cap, long long *out_len,
                                  int32_t *stk)
{
    Ctl *c = P.ctl;
    if (c->status != 0) { *out_len = 0; return; }
    const int32_t *ar = P.tab + P.tab[4];
    long long n = 0, sp = 0;
    stk[sp++] = 1;
    while (sp > 0) {
        const int32_t x = stk[--sp];
        const int32_t s = hs_at(P, x);
        if (n >= out_cap) { c->status = TRS_ERR_BUFFER_SMALL; *out_len = -1; return; }
        out[n++] = s;
        for (int a = (ar[s] & 0xff) - 1; a >= 0; a--) {
            if (sp >= P.cap) { c->status = TRS_ERR_BUFFER_SMALL; *out_len = -1; return; }
            stk[sp++] = arg_at(P, a, x);
        }
    }
    *out_len = n;
}

int fail(const std::string &m, int code)
{
    set_error(m);
    return code;
}

}  // namespace
}  // namespace trs

using namespace trs;

extern "C" int trs_normalize_static(const trs_program *prog, const int32_t *d_term, int64_t len,
                                    int32_t *d_out, int64_t out_cap, int64_t *d_out_len,
                                    const trs_opts *opts, trs_stats *stats, trs_stream stream)
{
    if (!prog || !d_term || !d_out || !d_out_len || len <= 0 || out_cap < 0)
        return fail("trs_normalize_static: bad argument", TRS_ERR_ARG);
    trs_opts o;
    if (opts) o = *opts;
    else trs_opts_default(&o);
    if (o.mode == TRS_MODE_LEARNED || o.driver != TRS_DRIVER_PERSISTENT || o.block_size < 128 ||
        o.block_size > 512 || (o.block_size & (o.block_size - 1)) || o.max_sweeps <= 0 ||
        o.timeout_ns <= 0 || o.time_limit_ns <= 0 || o.gc_div < 0 || o.gc_min_dead < 0 ||
        o.solo_max < 0 || o.grid_blocks < 0)
        return fail("trs_normalize_static: invalid options (plain or frontier mode, persistent driver)",
                    TRS_ERR_ARG);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail("trs_normalize_static: no usable current device", TRS_ERR_CUDA);
    unsigned char *base = nullptr;
    {
        // set-up, once per device (with that device current): the device
        // address of the file-scope array
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess)
                return fail(std::string("trs_normalize_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e),
                            TRS_ERR_CUDA);
            g_addr[dev] = (unsigned char *)p;
        }
        base = g_addr[dev];
    }
    const Program &p = prog->p;
    DevPool d{};
    const long long cap = carve(base, p, &d);
    if (cap < 2) return fail("trs_normalize_static: rule tables do not fit the static array", TRS_ERR_TOO_BIG);
    if (len + 1 > cap)
        return fail("trs_normalize_static: term of " + std::to_string(len) + " symbols exceeds the " +
                    std::to_string(cap - 1) + "-slot static node store", TRS_ERR_TOO_BIG);
    int sms = 0, bps = 0;
    // the engine specialised to the program's rules, when there is one
    const void *fn = (!o.generic && prog->spec) ? spec_kernel(prog->spec, o.mode) : nullptr;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = engine_configure(o.mode, o.block_size, engine_smem_bytes(d, o.mode, o.block_size), &bps, fn);
    if (e != cudaSuccess || bps <= 0) return fail("trs_normalize_static: occupancy query failed", TRS_ERR_CUDA);
    LaunchOpts lo{};
    lo.mode = o.mode;
    lo.block = o.block_size;
    lo.grid = o.grid_blocks > 0 ? std::min(o.grid_blocks, bps * sms) : bps * sms;
    lo.gc_min_dead = o.gc_min_dead;
    lo.gc_div = o.gc_div;
    lo.solo_max = o.solo_max;
    lo.trace = 0;
    lo.refresh = o.refresh;
    lo.threshold = o.threshold;
    lo.timeout_ns = o.timeout_ns;
    lo.time_limit_ns = o.time_limit_ns;
    // clear the control block, every stamp and the candidate bitmap (a
    // previous call leaves stamps and bits above this term's slots, and the
    // engine hands slots above the high-water mark back to the free ring as
    // free, stamp 0, without writing them), copy the rule table, build,
    // normalise, serialise
    e = cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.nfs, 0, (size_t)cap * sizeof(int32_t), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.dbm, 0, (size_t)(cap + 31) / 32 * sizeof(uint32_t), stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)d.tab, p.table.data(), p.table.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return fail(std::string("trs_normalize_static: ") + cudaGetErrorString(e), TRS_ERR_CUDA);
    e = prep_launch(d.ctl, o.max_sweeps, o.mode != TRS_MODE_PLAIN ? 1 : 0, stream);
    if (e != cudaSuccess) return fail(std::string("trs_normalize_static: ") + cudaGetErrorString(e), TRS_ERR_CUDA);
    // a malformed term sets the status word; the engine and the download then
    // do nothing
    k_static_upload<<<1, 1, 0, stream>>>(d, d_term, len, d.fq[0], d.fq[1]);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = engine_launch(d, lo, LLONG_MAX, 0ull, stream, fn);
    if (e != cudaSuccess) return fail(std::string("trs_normalize_static: ") + cudaGetErrorString(e), TRS_ERR_CUDA);
    k_static_download<<<1, 1, 0, stream>>>(d, d_out, out_cap, (long long *)d_out_len, d.fq[0]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(std::string("trs_normalize_static: ") + cudaGetErrorString(e), TRS_ERR_CUDA);
    Ctl h;
    e = cudaMemcpyAsync(&h, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(std::string("trs_normalize_static: ") + cudaGetErrorString(e), TRS_ERR_CUDA);
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->status = h.status;
        stats->rewrites = h.st_rewrites;
        stats->nf_marks = h.st_nf_marks;
        stats->sweeps = h.st_sweeps;
        stats->visits = h.st_visits;
        stats->allocs = h.st_allocs;
        stats->frees = h.st_frees;
        stats->gc_runs = h.st_gc_runs;
        stats->confirm_sweeps = h.st_confirm;
        stats->confirm_found = h.st_confirm_found;
        stats->frontier_peak = h.st_frontier_peak;
        stats->high_water = h.n_top;
        stats->solo_sweeps = h.st_solo_sweeps;
        stats->specialised = fn != nullptr;
    }
    if (h.status != 0) return fail("trs_normalize_static: device status " + std::to_string(h.status), h.status);
    set_error("");
    return TRS_OK;
}
