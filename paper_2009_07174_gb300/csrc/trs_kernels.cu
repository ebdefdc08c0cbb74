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

#include "trs_device.cuh"

namespace trs {

struct Flags {
    bool done, gc, confirm, stop;
};

__device__ __forceinline__ State load_state(const Ctl *ctl)
{
    State S;
    S.k = ldcg_s64(&ctl->sweep_id);
    S.n = ldcg_s64(&ctl->n_top);
    S.fb = ldcg_s64(&ctl->fl_begin);
    S.fe = ldcg_s64(&ctl->fl_end);
    S.dead = ldcg_s64(&ctl->dead);
    S.fsz = ldcg_s64(&ctl->fq_size);
    S.left = ldcg_s64(&ctl->sweeps_left);
    S.cur = __ldcg(&ctl->fq_cur);
    return S;
}

__device__ __forceinline__ void store_state(Ctl *ctl, const State &S)
{
    ctl->sweep_id = S.k;
    ctl->n_top = S.n;
    ctl->fl_begin = S.fb;
    ctl->fl_end = S.fe;
    ctl->dead = S.dead;
    ctl->fq_size = S.fsz;
    ctl->sweeps_left = S.left;
    ctl->fq_cur = S.cur;
}

// Loop state after sweep S.k from its accumulator (Sec. 3 main loop: n grows
// by the fresh indices handed out; the loop ends after a sweep that changed
// nothing).  Pure function of (S, A): every block computes the same result.
__device__ Flags end_sweep(State &S, const Acc *A, const LaunchOpts &o, long long cap,
                           bool write_stats, Ctl *ctl, const DevPool &P)
{
    Flags F{false, false, false, false};
    unsigned long long rew = ldcg_u64(&A->rewrites), nfm = ldcg_u64(&A->nf_marks);
    unsigned long long vis = ldcg_u64(&A->visits), alc = ldcg_u64(&A->allocs);
    unsigned long long claims = ldcg_u64(&A->fl_claims), fresh = ldcg_u64(&A->fresh);
    unsigned long long deaths = ldcg_u64(&A->deaths), pushes = ldcg_u64(&A->pushes);
    S.n += (long long)fresh;
    S.fb = S.fb + (long long)claims < S.fe ? S.fb + (long long)claims : S.fe;
    S.dead += (long long)deaths;
    const bool action = rew + nfm > 0;
    if (write_stats) {
        ctl->st_rewrites += (long long)rew;
        ctl->st_nf_marks += (long long)nfm;
        ctl->st_visits += (long long)vis;
        ctl->st_allocs += (long long)alc;
        if (action) ctl->st_sweeps += 1;
        if (o.trace && action) {
            long long t = ctl->trace_n++;
            trs_sweep_record &rec = P.trace[t % P.trace_cap];
            rec.sweep = S.k;
            rec.rewrites = (int32_t)rew;
            rec.nf_marks = (int32_t)nfm;
            rec.visits = (int32_t)vis;
            rec.allocs = (int32_t)alc;
            rec.high_water = S.n;
        }
    }
    if (o.mode == M_PLAIN) {
        if (!action) { F.done = true; return F; }
    }
    S.k += 1;
    S.left -= 1;
    if (o.mode != M_PLAIN) {
        S.cur ^= 1;
        S.fsz = (long long)pushes;
        if (write_stats && S.fsz > ctl->st_frontier_peak) ctl->st_frontier_peak = S.fsz;
        if (S.fsz == 0) F.confirm = true;
    }
    long long thr = (long long)o.gc_min_dead;
    long long frac = S.n / (o.gc_div > 0 ? o.gc_div : 8);
    if (frac > thr) thr = frac;
    if (S.dead > 0 && (S.dead >= thr || S.n > cap - cap / 16)) F.gc = true;
    if (S.left <= 0 && !F.confirm) {
        if (write_stats) atomicCAS(&ctl->status, 0, TRS_ERR_SWEEP_LIMIT);
        F.stop = true;
    }
    // wall-clock limit of the whole call (a TRS may loop without allocating)
    if (write_stats && now_ns() - ctl->t_start > o.time_limit_ns) atomicCAS(&ctl->status, 0, TRS_ERR_TIMEOUT);
    return F;
}

__global__ void __launch_bounds__(1024)
k_engine(DevPool P, LaunchOpts o, long long budget, unsigned long long cond)
{
    extern __shared__ int32_t smem[];
    Ctl *ctl = P.ctl;
    if (__ldcg(&ctl->done) || __ldcg(&ctl->status) != 0) {
        // nothing left to do: end the graph loop too
        if (cond && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0);
        return;
    }
    const Tab T = stage_table(P, smem);
    State S = load_state(ctl);
    const bool b0 = blockIdx.x == 0, t0 = b0 && threadIdx.x == 0;
    const unsigned nblocks = gridDim.x;
    const long long wpb = blockDim.x >> 5;
    const long long gw0 = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
    const long long gnw = (long long)gridDim.x * wpb;
    unsigned solo_gen = __ldcg(&ctl->solo_gen);
    bool finished = false;
    // every block has read solo_gen before block 0 can start a solo episode
    if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;

    // initial frontier (frontier / learned modes): one full seed scan
    if (o.mode != M_PLAIN && __ldcg(&ctl->mode_phase) == 1) {
        phase_seed(P, T, S, &ctl->acc[S.k % 3], blockIdx.x, gridDim.x);
        if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
        S.fsz = (long long)ldcg_u64(&ctl->acc[S.k % 3].conf_found);
        if (t0) {
            ctl->mode_phase = 0;
            if (S.fsz > ctl->st_frontier_peak) ctl->st_frontier_peak = S.fsz;
        }
        if (S.fsz == 0) { finished = true; goto out; }
    }

    for (long long ran = 0; ran < budget;) {
        Flags F;
        const bool solo = o.mode != M_PLAIN && o.solo_max > 0 && S.fsz > 0 && S.fsz <= o.solo_max;
        if (solo) {
            // ---- solo episode: block 0 sweeps alone with block barriers, the
            // other blocks wait for it (bounded wait)
            if (b0) {
                __shared__ int s_stop;
                long long mine = 0;
                for (;;) {
                    if (threadIdx.x == 0) memset(&ctl->acc[(S.k + 1) % 3], 0, sizeof(Acc));
                    __syncthreads();
                    Acc *A = &ctl->acc[S.k % 3];
                    phase_frontier(P, T, S, A, o.mode, threadIdx.x >> 5, wpb);
                    __syncthreads();
                    F = end_sweep(S, A, o, P.cap, threadIdx.x == 0, ctl, P);
                    mine++;
                    if (threadIdx.x == 0) {
                        ctl->st_solo_sweeps += 1;
                        s_stop = ld_relaxed_s32(&ctl->status) != 0;
                    }
                    __syncthreads();
                    if (s_stop) F.stop = true;
                    if (F.done || F.gc || F.confirm || F.stop || S.fsz > o.solo_max || S.fsz == 0 ||
                        ran + mine >= budget)
                        break;
                }
                if (threadIdx.x == 0) {
                    store_state(ctl, S);
                    ctl->solo_flags = (int)F.done | ((int)F.gc << 1) | ((int)F.confirm << 2) |
                                      ((int)F.stop << 3);
                    ctl->solo_ran = mine;
                    __threadfence();
                    red_release_add_u32(&ctl->solo_gen, 1u);
                }
                __syncthreads();
            } else {
                __shared__ int s_ok;
                if (threadIdx.x == 0) {
                    long long tw = now_ns();
                    int ok = 1;
                    while (ld_acquire_u32(&ctl->solo_gen) == solo_gen) {
                        if (ld_relaxed_s32(&ctl->status) != 0) { ok = 0; break; }
                        if (now_ns() - tw > o.timeout_ns) { set_status(ctl, TRS_ERR_TIMEOUT); ok = 0; break; }
                        __nanosleep(200);
                    }
                    __threadfence();
                    s_ok = ok;
                }
                __syncthreads();
                if (!s_ok) goto out;
            }
            solo_gen++;
            S = load_state(ctl);
            const int fl = __ldcg(&ctl->solo_flags);
            F.done = fl & 1;
            F.gc = (fl >> 1) & 1;
            F.confirm = (fl >> 2) & 1;
            F.stop = (fl >> 3) & 1;
            ran += ldcg_s64(&ctl->solo_ran);
            if (F.done) { finished = true; goto out; }
            if (F.stop || __ldcg(&ctl->status) != 0) goto out;
        } else {
            // ---- one grid-wide sweep
            if (t0) memset(&ctl->acc[(S.k + 1) % 3], 0, sizeof(Acc));
            Acc *A = &ctl->acc[S.k % 3];
            if (o.mode == M_PLAIN) phase_plain(P, T, S, A, gw0, gnw);
            else phase_frontier(P, T, S, A, o.mode, gw0, gnw);
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            F = end_sweep(S, A, o, P.cap, t0, ctl, P);
            ran++;
            if (F.done) { finished = true; goto out; }
            if (F.stop) goto out;
        }
        // ---- garbage collection between sweeps
        if (F.gc) {
            Acc *A = &ctl->acc[S.k % 3];
            phase_gc(P, T, S, A, blockIdx.x, gridDim.x);
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            S.fe += (long long)ldcg_u64(&A->gc_append);
            S.dead += (long long)ldcg_u64(&A->gc_deaths) - (long long)ldcg_u64(&A->gc_frees);
            if (t0) {
                ctl->st_gc_runs += 1;
                ctl->st_frees += (long long)ldcg_u64(&A->gc_frees);
                ctl->gc_pending = 0;
            }
        }
        // ---- full confirmation sweep when the frontier ran dry
        if (F.confirm) {
            Acc *A = &ctl->acc[S.k % 3];
            phase_seed(P, T, S, A, blockIdx.x, gridDim.x);
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            S.fsz = (long long)ldcg_u64(&A->conf_found);
            if (t0) {
                ctl->st_confirm += 1;
                ctl->st_confirm_found += S.fsz;
                ctl->mode_phase = 0;
            }
            if (S.fsz == 0) { finished = true; goto out; }
            if (S.left <= 0) {
                if (t0) atomicCAS(&ctl->status, 0, TRS_ERR_SWEEP_LIMIT);
                goto out;
            }
        }
    }
out:
    if (t0) {
        store_state(ctl, S);
        if (finished) ctl->done = 1;
        if (cond && (finished || ld_relaxed_s32(&ctl->status) != 0))
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0);
    }
}

// Unpin a root (term_release).
__global__ void k_release(DevPool P, int32_t root)
{
    if (atomicSub(&P.rc[root], 1) == 1) atomicAdd((unsigned long long *)&P.ctl->dead, 1ull);
}

// Slot 0 is the null node: never live, never free-listed.
__global__ void k_reset(DevPool P)
{
    Ctl *c = P.ctl;
    c->sweep_id = 1;
    c->n_top = 1;
    P.hs[0] = 0;
    P.nfs[0] = 0;
    P.rc[0] = 0;
    P.par[0] = 0;
    P.pend[0] = 0;
}

// ---------------------------------------------------------------------------
// host-side launch helpers (called from trs_api.cu)

size_t engine_smem_bytes(const DevPool &P) { return (size_t)P.tab_words * sizeof(int32_t); }

cudaError_t engine_configure(int block, size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_engine, block, smem);
}

cudaError_t engine_launch(const DevPool &P, const LaunchOpts &o, long long budget,
                          unsigned long long cond, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)o.grid);
    cfg.blockDim = dim3((unsigned)o.block);
    cfg.dynamicSmemBytes = engine_smem_bytes(P);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_engine, P, o, budget, cond);
}

cudaError_t release_launch(const DevPool &P, int32_t root, cudaStream_t stream)
{
    k_release<<<1, 1, 0, stream>>>(P, root);
    return cudaGetLastError();
}

cudaError_t reset_launch(const DevPool &P, cudaStream_t stream)
{
    k_reset<<<1, 1, 0, stream>>>(P);
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
    c->t_start = now_ns();
}

cudaError_t prep_launch(Ctl *ctl, long long max_sweeps, int seed, cudaStream_t stream)
{
    k_prep<<<1, 1, 0, stream>>>(ctl, max_sweeps, seed);
    return cudaGetLastError();
}

void *engine_kernel_ptr() { return (void *)k_engine; }

}  // namespace trs
