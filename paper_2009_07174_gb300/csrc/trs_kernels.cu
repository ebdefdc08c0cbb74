// trs_kernels.cu -- the sweep loop.  One cooperative kernel, k_engine, runs up
// to `budget` sweeps and serves every driver:
//   persistent: one launch runs the whole normalisation (budget unlimited);
//   graph:      the body of a CUDA-graph while-loop; the kernel clears the
//               loop condition when the normalisation ends;
//   host:       one launch per sweep, the host reads the loop state back after
//               each (the main loop of Sec. 3).
// Between sweeps the blocks meet at a timed grid barrier; every block derives
// the next loop state from the same sweep accumulators, so no block has to
// broadcast decisions.  Frontier sweeps small enough for one block run on
// block 0 alone with only block-level barriers ("solo" episodes).
#include <cuda_runtime.h>

#include "trs_engine_kernel.cuh"

namespace trs {

// Unpin a root (term_release): the root becomes a collection candidate, and
// the next collection frees the term if that was its last reference.
__global__ void k_release(DevPool P, int32_t root)
{
    if (atomicSub(&rc_at(P, root), 1) == 1) {
        P.dbm[root >> 5] |= 1u << (root & 31);
        P.ctl->dead += 1;
    }
}

// Slot 0 is the null node: never live, never free-listed.  The candidate
// bitmap starts empty.
__global__ void k_reset(DevPool P)
{
    Ctl *c = P.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->sweep_id = 1;
        c->n_top = 1;
        for (int w = 0; w < P.rs; w++) P.rec[w] = 0;
        P.nfs[0] = 0;
    }
    const long long nw = (P.cap + 31) / 32;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < nw; w += (long long)gridDim.x * blockDim.x)
        P.dbm[w] = 0;
}

// ---------------------------------------------------------------------------
// host-side launch helpers (called from trs_api.cu)

static void *engine_fn(int mode)
{
    if (mode == M_PLAIN) return (void *)k_engine<M_PLAIN>;
    if (mode == M_FRONTIER) return (void *)k_engine<M_FRONTIER>;
    return (void *)k_engine<M_LEARNED>;
}

size_t engine_smem_bytes(const DevPool &P, int mode, int block)
{
    (void)mode;
    (void)block;
    return mlp_up16((size_t)P.tab_words * sizeof(int32_t)) + (P.mlp ? (size_t)P.mlp_bytes : 0);
}

// fn: the kernel to run (a specialised engine's), or nullptr for this file's
cudaError_t engine_configure(int mode, int block, size_t smem, int *blocks_per_sm, const void *fn)
{
    if (!fn) fn = engine_fn(mode);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

cudaError_t engine_launch(const DevPool &P, const LaunchOpts &o, long long budget,
                          unsigned long long cond, cudaStream_t stream, const void *fn)
{
    if (!fn) fn = engine_fn(o.mode);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)o.grid);
    cfg.blockDim = dim3((unsigned)o.block);
    cfg.dynamicSmemBytes = engine_smem_bytes(P, o.mode, o.block);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DevPool p = P;
    LaunchOpts oo = o;
    long long b = budget;
    unsigned long long c = cond;
    void *args[4] = {&p, &oo, &b, &c};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t release_launch(const DevPool &P, int32_t root, cudaStream_t stream)
{
    k_release<<<1, 1, 0, stream>>>(P, root);
    return cudaGetLastError();
}

cudaError_t reset_launch(const DevPool &P, cudaStream_t stream)
{
    k_reset<<<256, 256, 0, stream>>>(P);
    return cudaGetLastError();
}

}  // namespace trs

namespace trs {

// Reset the per-call part of the control block before a normalisation.
__global__ void k_prep(Ctl *c, long long max_sweeps, int seed)
{
    memset(c->acc, 0, sizeof(c->acc));
    c->done = 0;
    c->status = 0;
    c->gc_pending = 0;
    c->mode_phase = seed;
    c->solo_flags = 0;
    c->solo_ran = 0;
    c->sweeps_left = max_sweeps;
    c->fq_size = 0;
    c->fq_cur = 0;
    c->st_rewrites = c->st_nf_marks = c->st_sweeps = c->st_visits = c->st_allocs = 0;
    c->st_frees = c->st_gc_runs = c->st_confirm = c->st_confirm_found = 0;
    c->st_refreshes = c->st_frontier_peak = c->st_solo_sweeps = 0;
    c->trace_n = 0;
    c->bar_count = 0;
    c->since = 0;
    c->samp_n = 0;
    c->t_start = now_ns();
}

cudaError_t prep_launch(Ctl *ctl, long long max_sweeps, int seed, cudaStream_t stream)
{
    k_prep<<<1, 1, 0, stream>>>(ctl, max_sweeps, seed);
    return cudaGetLastError();
}

void *engine_kernel_ptr(int mode) { return engine_fn(mode); }

// Graph driver: clear the while-loop condition once the normalisation has
// ended or failed.  A node of its own after the engine kernel, so that the
// engines compiled at run time (which cannot call the device runtime) share
// the graph driver.
__global__ void k_graph_cond(DevPool P, unsigned long long cond)
{
    const Ctl *ctl = P.ctl;
    if (__ldcg(&ctl->done) || __ldcg(&ctl->status) != 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0);
}

void *graph_cond_ptr() { return (void *)k_graph_cond; }

}  // namespace trs
