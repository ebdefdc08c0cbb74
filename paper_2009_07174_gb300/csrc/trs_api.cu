// trs_api.cu -- the C ABI (include/trs.h): node-store pools in caller-owned
// device memory, term upload / download, and the three sweep-loop drivers.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "trs_engine.h"

namespace trs {
// trs_kernels.cu
size_t engine_smem_bytes(const DevPool &P, int mode, int block);
cudaError_t engine_configure(int mode, int block, size_t smem, int *blocks_per_sm, const void *fn = nullptr);
cudaError_t engine_launch(const DevPool &P, const LaunchOpts &o, long long budget,
                          unsigned long long cond, cudaStream_t stream,
                          const void *fn = nullptr);
cudaError_t release_launch(const DevPool &P, int32_t root, cudaStream_t stream);
cudaError_t reset_launch(const DevPool &P, cudaStream_t stream);
cudaError_t prep_launch(Ctl *ctl, long long max_sweeps, int seed, cudaStream_t stream);
void *engine_kernel_ptr(int mode);
void *graph_cond_ptr();
const unsigned char *predictor_block(const trs_predictor *p);
size_t predictor_block_bytes(const trs_predictor *p);
const trs_program *predictor_program(const trs_predictor *p);
// trs_transfer.cu
size_t upload_aux_bytes(long long total, long long nterms);
int device_upload(const DevPool &P, const int32_t *flat, const int64_t *offsets, long long nterms, long long base,
                  int32_t stamp, int32_t *d_flat, int32_t *d_e, int32_t *d_par, void *aux, int num_sms,
                  cudaStream_t s, cudaError_t *cuda_err);
int device_download(const DevPool &P, long long n_top, const int32_t *roots, int nroots, int32_t *buf,
                    int64_t cap, int64_t *offsets_out, void *scratch, size_t scratch_bytes, int num_sms,
                    long long limit_ns, cudaStream_t s, cudaError_t *cuda_err);
}  // namespace trs

using namespace trs;

struct GraphCache {
    bool valid = false;
    LaunchOpts key{};
    long long budget = 0;
    const unsigned char *mlp = nullptr;
    const void *fn = nullptr;  // engine kernel of the graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct trs_pool {
    const trs_program *prog = nullptr;
    DevPool d{};
    void *mem = nullptr;
    size_t bytes = 0;
    int device = 0;
    int num_sms = 0;
    GraphCache graph;
    LaunchOpts last{};
    int last_driver = 0;
    int last_spec = 0;      // the last normalisation ran a specialised engine
    int32_t *act = nullptr;              // per-slot act[] (predictor traces)
    const trs_predictor *pred = nullptr; // learned mode
};

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kHostWalkBytes = 16u << 20;            // records walked on the host up to this size
constexpr int64_t kDeviceUploadMin = 1 << 16;           // batches from this many symbols build on the device
constexpr long long kWalkLimitNs = 30LL * 1000 * 1000 * 1000;  // device walks give up after this

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t rec, nfs, ring, fq0, fq1, act, cand, dbm, trace, ctl, tab, total;
};

Layout layout(const Program &p, int64_t cap)
{
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes); return at; };
    const size_t slots = (size_t)cap * sizeof(int32_t);
    L.rec = take(slots * (size_t)rec_stride(p.maxarity));
    L.nfs = take(slots);
    L.ring = take(slots);
    L.fq0 = take(slots);
    L.fq1 = take(slots);
    L.act = take(slots);
    L.cand = take(slots);
    L.dbm = take(((size_t)cap + 31) / 32 * sizeof(uint32_t));
    L.trace = take(sizeof(trs_sweep_record) * (size_t)kTraceCap);
    L.ctl = take(sizeof(Ctl));
    L.tab = take(p.table.size() * sizeof(int32_t));
    L.total = off;
    return L;
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return TRS_ERR_CUDA;
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

int read_ctl(trs_pool *pool, Ctl *h, cudaStream_t stream)
{
    CK(cudaMemcpyAsync(h, pool->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream), "read control block");
    CK(cudaStreamSynchronize(stream), "stream synchronize");
    return TRS_OK;
}

// Validate one ground term in preorder; returns its length or -1.
bool valid_term(const Program &p, const int32_t *t, int64_t len)
{
    if (!t || len <= 0) return false;
    int64_t need = 1;
    for (int64_t i = 0; i < len; i++) {
        if (need == 0) return false;
        int32_t s = t[i];
        if (s <= 0 || s >= p.nsym) return false;
        need += p.arity[s] - 1;
    }
    return need == 0;
}

}  // namespace

extern "C" {

void trs_opts_default(trs_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = TRS_MODE_PLAIN;
    o->driver = TRS_DRIVER_PERSISTENT;
    o->block_size = 512;
    o->grid_blocks = 0;
    o->max_sweeps = 1LL << 40;
    o->timeout_ns = 10LL * 1000 * 1000 * 1000;
    o->gc_min_dead = 4096;
    o->gc_div = 0;
    o->solo_max = 0;
    o->graph_unroll = 16;
    o->refresh = 64;
    o->threshold = 0.5f;
    o->trace = 0;
    o->time_limit_ns = 120LL * 1000 * 1000 * 1000;
}

int trs_pool_bytes(const trs_program *prog, int64_t capacity, size_t *bytes)
{
    if (!prog || !bytes || capacity < 2 || capacity > TRS_MAX_CAPACITY) {
        set_error("trs_pool_bytes: bad argument");
        return TRS_ERR_ARG;
    }
    *bytes = layout(prog->p, capacity).total;
    return TRS_OK;
}

int trs_pool_create(const trs_program *prog, int64_t capacity, void *dev_mem, size_t bytes,
                    trs_stream stream, trs_pool **out)
{
    if (!out) { set_error("trs_pool_create: out is NULL"); return TRS_ERR_ARG; }
    *out = nullptr;
    if (!prog || !dev_mem || capacity < 2 || capacity > TRS_MAX_CAPACITY ||
        ((uintptr_t)dev_mem % kAlign) != 0) {
        set_error("trs_pool_create: bad argument (program, memory, alignment or capacity)");
        return TRS_ERR_ARG;
    }
    const Program &p = prog->p;
    Layout L = layout(p, capacity);
    if (bytes < L.total) { set_error("trs_pool_create: memory smaller than trs_pool_bytes"); return TRS_ERR_ARG; }
    trs_pool *pool = new trs_pool;
    pool->prog = prog;
    pool->mem = dev_mem;
    pool->bytes = bytes;
    char *b = (char *)dev_mem;
    DevPool &d = pool->d;
    d.rec = (int32_t *)(b + L.rec);
    d.rs = rec_stride(p.maxarity);
    d.nfs = (int32_t *)(b + L.nfs);
    d.ring = (int32_t *)(b + L.ring);
    d.fq[0] = (int32_t *)(b + L.fq0);
    d.fq[1] = (int32_t *)(b + L.fq1);
    d.act = nullptr;
    pool->act = (int32_t *)(b + L.act);
    d.cand = (int32_t *)(b + L.cand);
    d.dbm = (uint32_t *)(b + L.dbm);
    d.trace = (trs_sweep_record *)(b + L.trace);
    d.ctl = (Ctl *)(b + L.ctl);
    d.tab = (const int32_t *)(b + L.tab);
    d.cap = capacity;
    d.ma = p.maxarity;
    d.tab_words = (int32_t)p.table.size();
    d.trace_cap = kTraceCap;
    d.nsym = p.nsym;
    cudaError_t e = cudaGetDevice(&pool->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pool->num_sms, cudaDevAttrMultiProcessorCount, pool->device);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)d.tab, p.table.data(), p.table.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) { delete pool; return cuda_fail(e, "trs_pool_create"); }
    *out = pool;
    int st = trs_pool_reset(pool, stream);
    if (st != TRS_OK) { delete pool; *out = nullptr; return st; }
    CK(cudaStreamSynchronize(stream), "trs_pool_create: synchronize");
    return TRS_OK;
}

void trs_pool_free(trs_pool *pool)
{
    if (!pool) return;
    if (pool->graph.exec) cudaGraphExecDestroy(pool->graph.exec);
    if (pool->graph.graph) cudaGraphDestroy(pool->graph.graph);
    delete pool;
}

int trs_pool_reset(trs_pool *pool, trs_stream stream)
{
    if (!pool) { set_error("trs_pool_reset: pool is NULL"); return TRS_ERR_ARG; }
    CK(cudaMemsetAsync(pool->d.ctl, 0, sizeof(Ctl), stream), "trs_pool_reset");
    CK(reset_launch(pool->d, stream), "trs_pool_reset: launch");
    return TRS_OK;
}

int term_upload_batch(trs_pool *pool, const int32_t *flat, const int64_t *offsets, int32_t nterms,
                      int32_t *roots_out, trs_stream stream)
{
    if (!pool || nterms < 0 || (nterms > 0 && (!flat || !offsets || !roots_out))) {
        set_error("term_upload_batch: bad argument");
        return TRS_ERR_ARG;
    }
    if (nterms == 0) return TRS_OK;
    const Program &p = pool->prog->p;
    for (int32_t t = 0; t < nterms; t++)
        if (offsets[t + 1] <= offsets[t]) {
            set_error("term_upload_batch: term " + std::to_string(t) + " is empty");
            return TRS_ERR_BAD_TERM;
        }
    const int64_t total = offsets[nterms] - offsets[0];
    Ctl h;
    int st = read_ctl(pool, &h, stream);
    if (st != TRS_OK) return st;
    const int64_t base = h.n_top;
    if (base + total > pool->d.cap) {
        set_error("term_upload_batch: pool full");
        return TRS_ERR_POOL_FULL;
    }
    const DevPool &d = pool->d;
    // Large batches are built on the device (trs_transfer.cu): only the
    // preorder symbols and offsets cross, the frontier buffers and the
    // predictor-trace array hold the per-symbol scratch, and the records of
    // the slots being filled hold the rest until they are written.
    const size_t rec_area = (size_t)total * d.rs * sizeof(int32_t);
    if (total >= kDeviceUploadMin && upload_aux_bytes(total, nterms) <= rec_area) {
        cudaError_t ce = cudaSuccess;
        st = device_upload(d, flat, offsets, nterms, base, -(int32_t)h.sweep_id, d.fq[0], d.fq[1], pool->act,
                           (void *)(d.rec + (size_t)base * d.rs), pool->num_sms, stream, &ce);
        if (st == TRS_ERR_CUDA) return cuda_fail(ce, "term_upload_batch (device build)");
        if (st == TRS_ERR_BAD_TERM) {
            set_error("term_upload_batch: the batch is not a sequence of well-formed ground terms");
            return st;
        }
        for (int32_t t = 0; t < nterms; t++) roots_out[t] = (int32_t)(base + offsets[t] - offsets[0]);
        long long ntop = base + total;
        CK(cudaMemcpyAsync(&d.ctl->n_top, &ntop, sizeof(ntop), cudaMemcpyHostToDevice, stream), "upload n_top");
        CK(cudaStreamSynchronize(stream), "upload synchronize");
        return TRS_OK;
    }
    for (int32_t t = 0; t < nterms; t++) {
        if (!valid_term(p, flat + offsets[t], offsets[t + 1] - offsets[t])) {
            set_error("term_upload_batch: term " + std::to_string(t) + " is not a ground term");
            return TRS_ERR_BAD_TERM;
        }
    }
    const int ma = p.maxarity, rs = rec_stride(ma);
    // records: head, arguments, parent word, count 1 (the tree edge or the
    // root's pin), pending 0 (set by the seed scan)
    std::vector<int32_t> rec((size_t)rs * total, 0), nfs(total, -(int32_t)h.sweep_id);
    struct Open { int64_t node; int32_t next, arity; };
    std::vector<Open> stk;
    for (int32_t t = 0; t < nterms; t++) {
        const int64_t b = offsets[t] - offsets[0];
        const int64_t len = offsets[t + 1] - offsets[t];
        stk.clear();
        for (int64_t q = 0; q < len; q++) {
            const int32_t s = flat[offsets[t] + q];
            const int64_t node = b + q;
            int32_t *r = &rec[(size_t)node * rs];
            r[kRecHead] = s;
            r[rec_rc(ma)] = 1;
            if (!stk.empty()) {
                Open &o = stk.back();
                rec[(size_t)o.node * rs + rec_arg(o.next)] = (int32_t)(base + node);
                // sign bit: the parent's head is unary (its only argument)
                r[rec_par(ma)] = (int32_t)((uint32_t)(base + o.node) | (o.arity == 1 ? 0x80000000u : 0u));
                if (++o.next == o.arity) stk.pop_back();
            }
            if (p.arity[s] > 0) stk.push_back({node, 0, p.arity[s]});
        }
        roots_out[t] = (int32_t)(base + b);
    }
    const size_t sz = (size_t)total * sizeof(int32_t);
    CK(cudaMemcpyAsync(d.rec + (size_t)base * rs, rec.data(), sz * rs, cudaMemcpyHostToDevice, stream),
       "upload records");
    CK(cudaMemcpyAsync(d.nfs + base, nfs.data(), sz, cudaMemcpyHostToDevice, stream), "upload nfs");
    long long ntop = base + total;
    CK(cudaMemcpyAsync(&d.ctl->n_top, &ntop, sizeof(ntop), cudaMemcpyHostToDevice, stream), "upload n_top");
    CK(cudaStreamSynchronize(stream), "upload synchronize");
    return TRS_OK;
}

int term_upload(trs_pool *pool, const int32_t *preorder, int64_t len, int32_t *root_out,
                trs_stream stream)
{
    int64_t offs[2] = {0, len};
    return term_upload_batch(pool, preorder, offs, 1, root_out, stream);
}

int term_release(trs_pool *pool, int32_t root, trs_stream stream)
{
    if (!pool || root <= 0 || root >= pool->d.cap) { set_error("term_release: bad argument"); return TRS_ERR_ARG; }
    CK(release_launch(pool->d, root, stream), "term_release");
    return TRS_OK;
}

static int validate_opts(const trs_opts *o)
{
    if (o->mode < 0 || o->mode > 2 || o->driver < 0 || o->driver > 2) return TRS_ERR_ARG;
    if (o->block_size != 128 && o->block_size != 256 && o->block_size != 512) return TRS_ERR_ARG;
    if (o->max_sweeps <= 0 || o->timeout_ns <= 0 || o->gc_div < 0 || o->gc_min_dead < 0 ||
        o->grid_blocks < 0 || o->solo_max < 0 || o->graph_unroll <= 0 || o->time_limit_ns <= 0 ||
        o->eager < 0 || o->generic < 0 || o->generic > 1)
        return TRS_ERR_ARG;
    return TRS_OK;
}

static bool same_key(const LaunchOpts &a, const LaunchOpts &b)
{
    return std::memcmp(&a, &b, sizeof(LaunchOpts)) == 0;
}

// Build (once per launch configuration) a graph whose only node is a while
// loop around the engine kernel; the kernel clears the loop condition when the
// normalisation ends or fails.
static int build_graph(trs_pool *pool, const DevPool &dp, const LaunchOpts &o, long long budget, const void *fn)
{
    GraphCache &G = pool->graph;
    if (G.valid && same_key(G.key, o) && G.budget == budget && G.mlp == dp.mlp && G.fn == fn) return TRS_OK;
    if (G.exec) { cudaGraphExecDestroy(G.exec); G.exec = nullptr; }
    if (G.graph) { cudaGraphDestroy(G.graph); G.graph = nullptr; }
    G.valid = false;
    CK(cudaGraphCreate(&G.graph, 0), "graph create");
    cudaGraphConditionalHandle handle;
    CK(cudaGraphConditionalHandleCreate(&handle, G.graph, 1, cudaGraphCondAssignDefault), "conditional handle");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    CK(cudaGraphAddNode(&loop, G.graph, nullptr, nullptr, 0, &cp), "conditional node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    DevPool P = dp;
    LaunchOpts lo = o;
    long long bud = budget;
    unsigned long long cond = (unsigned long long)handle;
    void *kargs[4] = {&P, &lo, &bud, &cond};
    cudaKernelNodeParams kp = {};
    kp.func = fn ? (void *)fn : engine_kernel_ptr(o.mode);
    kp.gridDim = dim3((unsigned)o.grid);
    kp.blockDim = dim3((unsigned)o.block);
    kp.sharedMemBytes = (unsigned)engine_smem_bytes(dp, o.mode, o.block);
    kp.kernelParams = kargs;
    cudaGraphNode_t kn;
    CK(cudaGraphAddKernelNode(&kn, body, nullptr, 0, &kp), "kernel node");
    cudaLaunchAttributeValue v = {};
    v.cooperative = 1;
    CK(cudaGraphKernelNodeSetAttribute(kn, cudaLaunchAttributeCooperative, &v), "cooperative attribute");
    // the loop condition is cleared by a one-thread kernel after the engine
    // (engines compiled at run time cannot call the device runtime)
    void *cargs[2] = {&P, &cond};
    cudaKernelNodeParams cq = {};
    cq.func = graph_cond_ptr();
    cq.gridDim = dim3(1);
    cq.blockDim = dim3(1);
    cq.kernelParams = cargs;
    cudaGraphNode_t cn;
    CK(cudaGraphAddKernelNode(&cn, body, &kn, 1, &cq), "condition node");
    CK(cudaGraphInstantiate(&G.exec, G.graph, 0), "graph instantiate");
    G.key = o;
    G.budget = budget;
    G.mlp = dp.mlp;
    G.fn = fn;
    G.valid = true;
    return TRS_OK;
}

int trs_normalize(trs_pool *pool, const trs_opts *opts, trs_stats *stats, trs_stream stream)
{
    if (!pool) { set_error("trs_normalize: pool is NULL"); return TRS_ERR_ARG; }
    trs_opts o;
    if (opts) o = *opts;
    else trs_opts_default(&o);
    if (validate_opts(&o) != TRS_OK) { set_error("trs_normalize: invalid options"); return TRS_ERR_ARG; }
    if (o.mode == TRS_MODE_LEARNED && !pool->pred) {
        set_error("trs_normalize: learned mode needs an attached predictor");
        return TRS_ERR_NO_PREDICTOR;
    }
    DevPool d = pool->d;
    if (o.mode == TRS_MODE_LEARNED) {
        d.mlp = predictor_block(pool->pred);
        d.mlp_bytes = (int32_t)predictor_block_bytes(pool->pred);
    }
    // the engine specialised to this program's rules, when there is one
    const void *fn = nullptr;
    if (!o.generic && pool->prog->spec) fn = spec_kernel(pool->prog->spec, o.mode);
    const size_t smem = engine_smem_bytes(d, o.mode, o.block_size);
    int bps = 0;
    CK(engine_configure(o.mode, o.block_size, smem, &bps, fn), "occupancy");
    if (bps <= 0) { set_error("trs_normalize: kernel does not fit on an SM"); return TRS_ERR_CUDA; }
    int max_grid = bps * pool->num_sms;
    int grid = o.grid_blocks > 0 ? std::min(o.grid_blocks, max_grid) : max_grid;
    LaunchOpts lo{};
    lo.mode = o.mode;
    lo.block = o.block_size;
    lo.grid = grid;
    lo.gc_min_dead = o.gc_min_dead;
    lo.gc_div = o.gc_div;
    lo.solo_max = o.solo_max;
    lo.trace = o.trace;
    lo.refresh = o.refresh;
    lo.threshold = o.threshold;
    lo.timeout_ns = o.timeout_ns;
    lo.time_limit_ns = o.time_limit_ns;
    lo.eager = o.mode != TRS_MODE_PLAIN ? o.eager : 0;
    pool->last = lo;
    pool->last_driver = o.driver;
    pool->last_spec = fn != nullptr;
    CK(prep_launch(pool->d.ctl, o.max_sweeps, o.mode != TRS_MODE_PLAIN ? 1 : 0, stream), "prepare");
    if (o.driver == TRS_DRIVER_PERSISTENT) {
        CK(engine_launch(d, lo, LLONG_MAX, 0ull, stream, fn), "engine launch");
    } else if (o.driver == TRS_DRIVER_GRAPH) {
        int st = build_graph(pool, d, lo, o.graph_unroll, fn);
        if (st != TRS_OK) return st;
        CK(cudaGraphLaunch(pool->graph.exec, stream), "graph launch");
    } else {
        // Sec. 3 main loop: launch one sweep, read the loop state back, repeat
        int hflags[2];
        for (;;) {
            CK(engine_launch(d, lo, 1, 0ull, stream, fn), "engine launch");
            CK(cudaMemcpyAsync(&hflags[0], &pool->d.ctl->done, sizeof(int), cudaMemcpyDeviceToHost, stream),
               "read done");
            CK(cudaMemcpyAsync(&hflags[1], &pool->d.ctl->status, sizeof(int), cudaMemcpyDeviceToHost, stream),
               "read status");
            CK(cudaStreamSynchronize(stream), "sweep synchronize");
            if (hflags[0] || hflags[1]) break;
        }
    }
    if (stats) return trs_pool_stats(pool, stats, stream);
    return TRS_OK;
}

int trs_pool_attach_predictor(trs_pool *pool, const trs_predictor *pred)
{
    if (!pool) { set_error("trs_pool_attach_predictor: pool is NULL"); return TRS_ERR_ARG; }
    if (pred && predictor_program(pred) != pool->prog) {
        set_error("trs_pool_attach_predictor: predictor built for another program");
        return TRS_ERR_ARG;
    }
    pool->pred = pred;
    return TRS_OK;
}

int trs_collect_samples(trs_pool *pool, const trs_opts *opts, int32_t period, float rate, uint64_t seed,
                        void *dev_samples, int64_t cap, int64_t *n_out, trs_stats *stats, trs_stream stream)
{
    if (!pool || !dev_samples || cap <= 0 || !n_out || period <= 0 || !(rate > 0.f) || rate > 1.f ||
        ((uintptr_t)dev_samples % 256) != 0) {
        set_error("trs_collect_samples: bad argument");
        return TRS_ERR_ARG;
    }
    trs_opts o;
    if (opts) o = *opts;
    else trs_opts_default(&o);
    if (validate_opts(&o) != TRS_OK || o.mode == TRS_MODE_LEARNED) {
        set_error("trs_collect_samples: invalid options (plain or frontier mode)");
        return TRS_ERR_ARG;
    }
    const Program &p = pool->prog->p;
    const int F = 2 + p.maxarity;
    DevPool d = pool->d;
    d.act = pool->act;
    d.samp_feat = (int32_t *)dev_samples;
    const size_t feat_b = ((size_t)cap * F * 4 + 255) / 256 * 256;
    d.samp_slot = (int32_t *)((char *)dev_samples + feat_b);
    d.samp_label = (float *)((char *)dev_samples + feat_b + ((size_t)cap * 4 + 255) / 256 * 256);
    d.samp_cap = cap;
    int bps = 0;
    const void *fn = nullptr;
    if (!o.generic && pool->prog->spec) fn = spec_kernel(pool->prog->spec, o.mode);
    CK(engine_configure(o.mode, o.block_size, engine_smem_bytes(d, o.mode, o.block_size), &bps, fn), "occupancy");
    if (bps <= 0) { set_error("trs_collect_samples: kernel does not fit on an SM"); return TRS_ERR_CUDA; }
    LaunchOpts lo{};
    lo.mode = o.mode;
    lo.block = o.block_size;
    lo.grid = o.grid_blocks > 0 ? std::min(o.grid_blocks, bps * pool->num_sms) : bps * pool->num_sms;
    lo.gc_min_dead = o.gc_min_dead;
    lo.gc_div = o.gc_div;
    lo.solo_max = 0;  // sampling sweeps are grid-wide and synchronous
    lo.eager = 0;
    lo.trace = o.trace;
    lo.timeout_ns = o.timeout_ns;
    lo.time_limit_ns = o.time_limit_ns;
    lo.sample_period = period;
    const double t = (double)rate * 4294967296.0;
    lo.sample_thresh = t >= 4294967295.0 ? 0xffffffffu : (uint32_t)t;
    lo.sample_seed = (uint32_t)(seed ^ (seed >> 32));
    CK(prep_launch(pool->d.ctl, o.max_sweeps, o.mode != TRS_MODE_PLAIN ? 1 : 0, stream), "prepare");
    CK(engine_launch(d, lo, LLONG_MAX, 0ull, stream, fn), "engine launch");
    Ctl h;
    int st = read_ctl(pool, &h, stream);
    if (st != TRS_OK) return st;
    *n_out = std::min<int64_t>(h.samp_n, cap);
    if (stats) return trs_pool_stats(pool, stats, stream);
    if (h.status != 0) { set_error("trs_collect_samples: device status " + std::to_string(h.status)); return h.status; }
    return TRS_OK;
}

int trs_pool_stats(trs_pool *pool, trs_stats *s, trs_stream stream)
{
    if (!pool || !s) { set_error("trs_pool_stats: bad argument"); return TRS_ERR_ARG; }
    Ctl h;
    int st = read_ctl(pool, &h, stream);
    if (st != TRS_OK) return st;
    std::memset(s, 0, sizeof(*s));
    s->status = h.status;
    s->rewrites = h.st_rewrites;
    s->nf_marks = h.st_nf_marks;
    s->sweeps = h.st_sweeps;
    s->visits = h.st_visits;
    s->allocs = h.st_allocs;
    s->frees = h.st_frees;
    s->gc_runs = h.st_gc_runs;
    s->confirm_sweeps = h.st_confirm;
    s->confirm_found = h.st_confirm_found;
    s->refreshes = h.st_refreshes;
    s->frontier_peak = h.st_frontier_peak;
    s->high_water = h.n_top;
    // slots in use, less the free ring and the dead nodes not yet collected
    s->live_nodes = (h.n_top - 1) - (h.fl_end - h.fl_begin) - h.dead;
    s->solo_sweeps = h.st_solo_sweeps;
    s->specialised = pool->last_spec;
    if (h.status != 0) {
        set_error(std::string("trs_normalize: device status ") + std::to_string(h.status));
        return h.status;
    }
    return TRS_OK;
}

int term_download_batch(trs_pool *pool, const int32_t *roots, int32_t nroots, int32_t *buf,
                        int64_t cap, int64_t *offsets_out, trs_stream stream)
{
    if (!pool || nroots < 0 || (nroots > 0 && (!roots || !offsets_out)) || cap < 0 || (cap > 0 && !buf)) {
        set_error("term_download: bad argument");
        return TRS_ERR_ARG;
    }
    if (nroots == 0) {
        if (offsets_out) offsets_out[0] = 0;
        return TRS_OK;
    }
    const Program &p = pool->prog->p;
    Ctl h;
    int st = read_ctl(pool, &h, stream);
    if (st != TRS_OK) return st;
    const int64_t n = h.n_top;
    const DevPool &d = pool->d;
    for (int32_t r = 0; r < nroots; r++)
        if (roots[r] <= 0 || roots[r] >= n) { set_error("term_download: root out of range"); return TRS_ERR_STATE; }
    const int rs = d.rs;
    // A store whose records below the high-water mark fit kHostWalkBytes is
    // copied back in one piece and walked on the host: for it that is cheaper
    // than the device pass.  Larger stores are serialised on the device
    // (trs_transfer.cu) in the frontier buffers and the predictor-trace array,
    // which hold nothing between normalisations; only the result crosses.
    if ((size_t)n * rs * sizeof(int32_t) > kHostWalkBytes) {
        char *scratch = (char *)d.fq[0];
        const size_t scratch_bytes = (size_t)((char *)d.cand - scratch);
        cudaError_t ce = cudaSuccess;
        st = device_download(d, n, roots, nroots, buf, cap, offsets_out, scratch, scratch_bytes, pool->num_sms,
                             kWalkLimitNs, stream, &ce);
        if (st == TRS_ERR_CUDA) return cuda_fail(ce, "term_download (device pass)");
        if (st == TRS_OK) return TRS_OK;
        if (st == TRS_ERR_BUFFER_SMALL) { set_error("term_download: buffer too small"); return st; }
        if (st == TRS_ERR_STATE) { set_error("term_download: a root is not live, or the store is corrupt"); return st; }
        if (st == TRS_ERR_TIMEOUT) { set_error("term_download: a walk ran out of time (corrupt store)"); return st; }
        // TRS_ERR_TOO_BIG: a subtree deeper than the device stacks; walk on the host
    }
    std::vector<int32_t> rec((size_t)n * rs);
    CK(cudaMemcpyAsync(rec.data(), d.rec, (size_t)n * rs * sizeof(int32_t), cudaMemcpyDeviceToHost, stream),
       "download records");
    CK(cudaStreamSynchronize(stream), "download synchronize");
    // a root is live while it is referenced (freed slots have count 0)
    for (int32_t r = 0; r < nroots; r++)
        if (rec[(size_t)roots[r] * rs + rec_rc(p.maxarity)] <= 0) {
            set_error("term_download: root is not live");
            return TRS_ERR_STATE;
        }
    int64_t out = 0;
    std::vector<int32_t> stk;
    offsets_out[0] = 0;
    for (int32_t r = 0; r < nroots; r++) {
        stk.clear();
        stk.push_back(roots[r]);
        while (!stk.empty()) {
            int32_t x = stk.back();
            stk.pop_back();
            if (x <= 0 || x >= n) { set_error("term_download: dangling index"); return TRS_ERR_STATE; }
            const int32_t *rr = &rec[(size_t)x * rs];
            int32_t s = rr[kRecHead];
            if (s <= 0 || s >= p.nsym) { set_error("term_download: corrupt node"); return TRS_ERR_STATE; }
            if (out < cap) buf[out] = s;
            out++;
            for (int a = p.arity[s] - 1; a >= 0; a--) stk.push_back(rr[rec_arg(a)]);
        }
        offsets_out[r + 1] = out;
    }
    if (out > cap) {
        set_error("term_download: buffer too small");
        return TRS_ERR_BUFFER_SMALL;
    }
    return TRS_OK;
}

int term_download(trs_pool *pool, int32_t root, int32_t *buf, int64_t cap, int64_t *len_out,
                  trs_stream stream)
{
    if (!len_out) { set_error("term_download: len_out is NULL"); return TRS_ERR_ARG; }
    int64_t offs[2] = {0, 0};
    int st = term_download_batch(pool, &root, 1, buf, cap, offs, stream);
    *len_out = offs[1];
    return st;
}

int trs_trace_read(trs_pool *pool, trs_sweep_record *buf, int64_t cap, int64_t *n_out, trs_stream stream)
{
    if (!pool || !n_out || cap < 0 || (cap > 0 && !buf)) { set_error("trs_trace_read: bad argument"); return TRS_ERR_ARG; }
    Ctl h;
    int st = read_ctl(pool, &h, stream);
    if (st != TRS_OK) return st;
    int64_t n = std::min<int64_t>(h.trace_n, kTraceCap);
    int64_t first = h.trace_n - n;
    int64_t take = std::min(n, cap);
    std::vector<trs_sweep_record> all(kTraceCap);
    CK(cudaMemcpyAsync(all.data(), pool->d.trace, sizeof(trs_sweep_record) * kTraceCap,
                       cudaMemcpyDeviceToHost, stream), "trace read");
    CK(cudaStreamSynchronize(stream), "trace read");
    for (int64_t i = 0; i < take; i++) buf[i] = all[(first + i) % kTraceCap];
    *n_out = n;
    return TRS_OK;
}

}  // extern "C"
