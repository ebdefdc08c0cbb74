// trs_engine_kernel.cuh -- the sweep loop kernel (k_engine) and its per-sweep
// bookkeeping.  Included by trs_kernels.cu (table-driven rule matching) and by
// the run-time compiled engine specialised to one rule system (trs_spec.cpp),
// so that both run the same loop.
#pragma once

#include "trs_device.cuh"

namespace trs {

struct Flags {
    bool done, gc, confirm, stop, refresh;
    bool stall;  // learned mode: the sweep changed nothing
};


struct AccVals {
    unsigned long long rew, nfm, vis, alc, claims, ret, deaths, pushes;
};

// Statistics of the running call, kept by thread 0 of block 0 and added to the
// control block when the launch ends.
struct LocalStats {
    long long rewrites, nf_marks, sweeps, visits, allocs, frees, gc_runs, confirm, confirm_found;
    long long frontier_peak, solo_sweeps, refreshes;
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
    S.since = ldcg_s64(&ctl->since);
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
    ctl->since = S.since;
    ctl->fq_cur = S.cur;
}

// One thread reads the sweep accumulator (from L2, or from shared memory in a
// solo episode) and the block shares it.
__device__ __forceinline__ AccVals read_acc(const Acc *A, bool in_smem)
{
    __shared__ AccVals s_v;
    if (threadIdx.x == 0) {
        AccVals v;
        if (in_smem) {
            const volatile Acc *a = A;
            v = AccVals{a->rewrites, a->nf_marks, a->visits, a->allocs, a->fl_claims, a->ret,
                        a->deaths, a->pushes};
        } else {
            v = AccVals{ldcg_u64(&A->rewrites), ldcg_u64(&A->nf_marks), ldcg_u64(&A->visits),
                        ldcg_u64(&A->allocs), ldcg_u64(&A->fl_claims), ldcg_u64(&A->ret),
                        ldcg_u64(&A->deaths), ldcg_u64(&A->pushes)};
        }
        s_v = v;
    }
    __syncthreads();
    AccVals v = s_v;
    __syncthreads();
    return v;
}

__device__ __forceinline__ unsigned long long read_u64_block(const unsigned long long *p)
{
    __shared__ unsigned long long s_x;
    if (threadIdx.x == 0) s_x = ldcg_u64(p);
    __syncthreads();
    unsigned long long x = s_x;
    __syncthreads();
    return x;
}

// Loop state after sweep S.k from its accumulator (Sec. 3 main loop: n grows
// by the fresh indices handed out; the loop ends after a sweep that changed
// nothing).  A pure function of (S, V): every block computes the same result.
__device__ Flags end_sweep(State &S, const AccVals &V, const LaunchOpts &o, long long cap)
{
    Flags F{false, false, false, false, false, false};
    // the sweep's allocation positions: the first `avail` were ring entries,
    // the rest fresh slots above the mark; unused ones came back behind fe
    const long long avail = S.fe - S.fb;
    const long long claims = (long long)V.claims;
    S.n += claims > avail ? claims - avail : 0;
    S.fb += claims < avail ? claims : avail;
    S.fe += (long long)V.ret;
    if (S.fb >= cap) {  // ring positions stay below 2 * cap
        S.fb -= cap;
        S.fe -= cap;
    }
    if (S.n > cap) S.n = cap;
    S.dead += (long long)V.deaths;
    const bool action = V.rew + V.nfm > 0;
    if (o.mode == M_PLAIN && !action) { F.done = true; return F; }
    S.k += 1;
    S.left -= 1;
    if (o.mode != M_PLAIN) {
        S.cur ^= 1;
        S.fsz = (long long)V.pushes;
        if (o.mode == M_FRONTIER && S.fsz == 0) F.confirm = true;
    }
    if (o.mode == M_LEARNED) {
        // re-score the whole store when the frontier ran dry, when a sweep
        // changed nothing, or every `refresh` sweeps
        S.since += 1;
        F.refresh = S.fsz == 0 || !action || S.since >= o.refresh;
        F.stall = !action;
    }
    // collection trigger: the plain sweep scans every slot below the high-water
    // mark, so it collects early (decrements >= n / 8 by default) to keep the
    // mark low; the frontier modes only pay for collection, so they collect
    // when the decrements reach the high-water mark itself (by default) or
    // when fewer than cap / 8 slots remain free (above the mark or in the ring)
    const int div = o.gc_div > 0 ? o.gc_div : (o.mode == M_PLAIN ? 8 : 1);
    long long thr = (long long)o.gc_min_dead;
    const long long frac = S.n / div;
    if (frac > thr) thr = frac;
    const long long free_slots = (cap - S.n) + (S.fe - S.fb);
    if (S.dead > 0 && (S.dead >= thr || free_slots < cap / 8)) F.gc = true;
    if (S.left <= 0 && !F.confirm && !F.refresh) F.stop = true;
    return F;
}

// Bookkeeping of thread 0 of block 0 after a sweep: statistics, trace record,
// sweep limit and wall-clock limit.
__device__ __forceinline__ void note_sweep(LocalStats &L, const AccVals &V, const State &S,
                                           const Flags &F, const LaunchOpts &o, Ctl *ctl,
                                           const DevPool &P, bool solo)
{
    const bool action = V.rew + V.nfm > 0;
    L.rewrites += (long long)V.rew;
    L.nf_marks += (long long)V.nfm;
    L.visits += (long long)V.vis;
    L.allocs += (long long)V.alc;
    if (action) L.sweeps++;
    if (solo) L.solo_sweeps++;
    if (o.mode != M_PLAIN && S.fsz > L.frontier_peak) L.frontier_peak = S.fsz;
    if (o.trace && action) {
        long long t = ctl->trace_n++;
        trs_sweep_record &rec = P.trace[t % P.trace_cap];
        rec.sweep = F.done ? S.k : S.k - 1;
        rec.rewrites = (int32_t)V.rew;
        rec.nf_marks = (int32_t)V.nfm;
        rec.visits = (int32_t)V.vis;
        rec.allocs = (int32_t)V.alc;
        rec.high_water = S.n;
        rec.t_ns = now_ns() - ctl->t_start;
        rec.frontier = (int32_t)(S.fsz < 0x7fffffff ? S.fsz : 0x7fffffff);
        rec.flags = (solo ? TRS_SWEEP_SOLO : 0) | (F.gc ? TRS_SWEEP_GC : 0) |
                    (F.confirm ? TRS_SWEEP_CONFIRM : 0) | (F.refresh ? TRS_SWEEP_REFRESH : 0);
    }
    if (F.stop) atomicCAS(&ctl->status, 0, TRS_ERR_SWEEP_LIMIT);
    if (now_ns() - ctl->t_start > o.time_limit_ns) atomicCAS(&ctl->status, 0, TRS_ERR_TIMEOUT);
}

// One instantiation per mode: the plain sweep needs few registers and gains
// from two resident blocks per SM; the frontier and learned paths get 128.
template <int MODE>
__global__ void __launch_bounds__(512, MODE == M_PLAIN ? 2 : 1)
k_engine(DevPool P, LaunchOpts o_in, long long budget, unsigned long long cond)
{
    LaunchOpts o = o_in;
    o.mode = MODE;
    extern __shared__ __align__(128) int32_t smem[];
    __shared__ Acc s_acc;
    __shared__ int s_flag;
    Ctl *ctl = P.ctl;
    if (__ldcg(&ctl->done) || __ldcg(&ctl->status) != 0) {
        // nothing left to do: end the graph loop too
#ifndef TRS_JIT
        if (cond && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0);
#endif
        return;
    }
    const Tab T = stage_table(P, smem);
    MlpView M{};
    if (o.mode == M_LEARNED && P.mlp) {
        unsigned char *mb = (unsigned char *)smem + mlp_up16((size_t)P.tab_words * 4);
        for (int t = threadIdx.x; t < P.mlp_bytes / 16; t += blockDim.x)
            reinterpret_cast<int4 *>(mb)[t] = reinterpret_cast<const int4 *>(P.mlp)[t];
        __syncthreads();
        M = mlp_view(mb, P.nsym, P.ma);
    }
    State S = load_state(ctl);
    const long long k_first = S.k;
    // predictor traces: the current batch of rows [s_lo, s_hi) and the sweep
    // it was sampled in; block-uniform, kept in shared memory (written by
    // thread 0 between barriers) so that it takes no registers
    __shared__ long long s_trace_rows[3];
    long long &s_lo = s_trace_rows[0], &s_hi = s_trace_rows[1], &s_k = s_trace_rows[2];
    if (threadIdx.x == 0) {
        s_lo = 0;
        s_hi = 0;
        s_k = -1;
    }
    const bool b0 = blockIdx.x == 0, t0 = b0 && threadIdx.x == 0;
    const unsigned nblocks = gridDim.x;
    const long long wpb = blockDim.x >> 5;
    const long long gw0 = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
    const long long gnw = (long long)gridDim.x * wpb;
    unsigned solo_gen = __ldcg(&ctl->solo_gen);
    bool finished = false;
    // statistics of this launch: kept by thread 0 of block 0 only, in shared
    // memory so that they occupy no registers in the sweep loop
    __shared__ LocalStats s_stats;
    LocalStats &L = s_stats;
    if (threadIdx.x == 0) L = LocalStats{};
    // seed requests are read by every block before anyone clears them
    const int phase0 = __ldcg(&ctl->mode_phase);
    // initial frontier, learned mode: a refresh scores the whole store
    bool start_refresh = o.mode == M_LEARNED && phase0 == 1;
    // every block has read solo_gen before block 0 can start a solo episode
    if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
    if (t0) ctl->mode_phase = 0;

    // initial frontier, frontier mode: one full seed scan
    if (o.mode == M_FRONTIER && phase0 == 1) {
        phase_seed(P, T, S, &ctl->acc[S.k % 3], blockIdx.x, gridDim.x);
        if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
        S.fsz = (long long)read_u64_block(&ctl->acc[S.k % 3].conf_found);
        if (t0 && S.fsz > L.frontier_peak) L.frontier_peak = S.fsz;
        if (S.fsz == 0) { finished = true; goto out; }
    }

    for (long long ran = 0; ran < budget;) {
        Flags F{false, false, false, false, false, false};
        const bool solo = o.mode != M_PLAIN && o.solo_max > 0 && S.fsz > 0 && S.fsz <= o.solo_max;
        if (start_refresh) {
            start_refresh = false;
            F.refresh = true;
        } else if (solo) {
            // ---- solo episode: block 0 sweeps alone with block barriers and
            // shared-memory accumulators; the other blocks wait (bounded)
            if (b0) {
                long long mine = 0;
                for (;;) {
                    if (threadIdx.x == 0) memset(&s_acc, 0, sizeof(Acc));
                    __syncthreads();
                    // the episode's frontier spread over the block's warps
                    long long per = (S.fsz + wpb - 1) / wpb;
                    if (per > 32) per = 32;
                    if (per < 1) per = 1;
                    phase_frontier(P, T, S, &s_acc, o.mode, threadIdx.x >> 5, wpb, o.eager, true, (int)per);
                    __syncthreads();
                    const AccVals V = read_acc(&s_acc, true);
                    F = end_sweep(S, V, o, P.cap);
                    mine++;
                    if (threadIdx.x == 0) {
                        note_sweep(L, V, S, F, o, ctl, P, true);
                        s_flag = ld_relaxed_s32(&ctl->status) != 0;
                    }
                    __syncthreads();
                    if (s_flag) F.stop = true;
                    if (F.done || F.gc || F.confirm || F.stop || F.refresh || S.fsz > o.solo_max ||
                        S.fsz == 0 || ran + mine >= budget)
                        break;
                }
                if (threadIdx.x == 0) {
                    // the grid phases that follow use the global accumulators
                    memset(&ctl->acc[S.k % 3], 0, sizeof(Acc));
                    memset(&ctl->acc[(S.k + 1) % 3], 0, sizeof(Acc));
                    store_state(ctl, S);
                    ctl->solo_flags = (int)F.done | ((int)F.gc << 1) | ((int)F.confirm << 2) |
                                      ((int)F.stop << 3) | ((int)F.refresh << 4) | ((int)F.stall << 5);
                    ctl->solo_ran = mine;
                    __threadfence();
                    red_release_add_u32(&ctl->solo_gen, 1u);
                }
                __syncthreads();
            } else {
                if (threadIdx.x == 0) {
                    long long tw = now_ns();
                    int ok = 1;
                    while (ld_relaxed_u32(&ctl->solo_gen) == solo_gen) {
                        if (ld_relaxed_s32(&ctl->status) != 0) { ok = 0; break; }
                        if (now_ns() - tw > o.timeout_ns) { set_status(ctl, TRS_ERR_TIMEOUT); ok = 0; break; }
                        __nanosleep(200);
                    }
                    __threadfence();
                    s_flag = ok;
                }
                __syncthreads();
                if (!s_flag) goto out;
            }
            solo_gen++;
            S = load_state(ctl);
            const int fl = __ldcg(&ctl->solo_flags);
            F.done = fl & 1;
            F.gc = (fl >> 1) & 1;
            F.confirm = (fl >> 2) & 1;
            F.stop = (fl >> 3) & 1;
            F.refresh = (fl >> 4) & 1;
            F.stall = (fl >> 5) & 1;
            ran += ldcg_s64(&ctl->solo_ran);
            if (F.done) { finished = true; goto out; }
            if (F.stop || __ldcg(&ctl->status) != 0) goto out;
        } else {
            // ---- predictor traces: label the previous rows, sample new ones
            if (P.samp_feat && o.sample_period > 0 && (S.k - k_first) % o.sample_period == 0) {
                if (s_k >= 0) phase_label(P, s_lo, s_hi, S.k);
                phase_sample(P, T, S, o);
                if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
                long long hi = (long long)read_u64_block((const unsigned long long *)&ctl->samp_n);
                if (hi > P.samp_cap) hi = P.samp_cap;
                if (threadIdx.x == 0) {
                    s_lo = s_hi;
                    s_hi = hi;
                    s_k = S.k;
                }
                __syncthreads();
            }
            // ---- one grid-wide sweep
            if (t0) memset(&ctl->acc[(S.k + 1) % 3], 0, sizeof(Acc));
            Acc *A = &ctl->acc[S.k % 3];
            if (o.mode == M_PLAIN) phase_plain(P, T, S, A, gw0, gnw);
            else {
                // busy lanes per warp: the frontier spread over every warp
                long long per = (S.fsz + gnw - 1) / gnw;
                if (o.eager <= 0 || per > 32) per = 32;
                if (per < 1) per = 1;
                phase_frontier(P, T, S, A, o.mode, gw0, gnw, o.eager, per == 1, (int)per);
            }
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            const AccVals V = read_acc(A, false);
            F = end_sweep(S, V, o, P.cap);
            if (t0) note_sweep(L, V, S, F, o, ctl, P, false);
            ran++;
            if (F.done) { finished = true; goto out; }
            if (F.stop) goto out;
        }
        // ---- garbage collection between sweeps
        if (F.gc) {
            Acc *A = &ctl->acc[S.k % 3];
            phase_gc_collect(P, S, A, gw0, gnw);
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            const long long ncand = (long long)read_u64_block(&A->gc_cand);
            phase_gc_free(P, T, S, A, ncand, gw0, gnw);
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            __shared__ unsigned long long s_gc[3];
            if (threadIdx.x == 0) {
                s_gc[0] = ldcg_u64(&A->gc_append);
                s_gc[1] = ldcg_u64(&A->gc_deaths);
                s_gc[2] = ldcg_u64(&A->gc_frees);
            }
            __syncthreads();
            S.fe += (long long)s_gc[0];
            // every candidate whose count was 0 was freed with the nodes it
            // killed; dead nodes the walks left are marked for the next one
            S.dead = (long long)s_gc[1];
            if (t0) {
                L.gc_runs += 1;
                L.frees += (long long)s_gc[2];
            }
            __syncthreads();
        }
        // ---- full confirmation sweep when the frontier ran dry
        if (F.confirm) {
            Acc *A = &ctl->acc[S.k % 3];
            phase_seed(P, T, S, A, blockIdx.x, gridDim.x);
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            S.fsz = (long long)read_u64_block(&A->conf_found);
            if (t0) {
                L.confirm += 1;
                L.confirm_found += S.fsz;
            }
            if (S.fsz == 0) { finished = true; goto out; }
            if (S.left <= 0) {
                if (t0) atomicCAS(&ctl->status, 0, TRS_ERR_SWEEP_LIMIT);
                goto out;
            }
        }
        // ---- learned frontier: re-score the store
        if (F.refresh) {
            Acc *A = &ctl->acc[S.k % 3];
            phase_refresh(P, T, M, S, A, o.threshold, blockIdx.x, gridDim.x);
            if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
            __shared__ unsigned long long s_rf[2];
            if (threadIdx.x == 0) {
                s_rf[0] = ldcg_u64(&A->refresh_sel);
                s_rf[1] = ldcg_u64(&A->pending);
            }
            __syncthreads();
            const long long sel = (long long)s_rf[0], pend = (long long)s_rf[1];
            __syncthreads();
            if (t0) {
                L.refreshes += 1;
                L.confirm += 1;
                if (sel > L.frontier_peak) L.frontier_peak = sel;
            }
            S.since = 0;
            if (pend == 0) { finished = true; goto out; }  // a full scan found no work
            S.fsz += sel;
            if (S.fsz == 0 || F.stall) {
                // nothing queued or selected, or the last frontier made no
                // progress (it may hold only nodes that wait for others, and
                // would be selected again): take the ready nodes instead
                phase_seed(P, T, S, A, blockIdx.x, gridDim.x, M_LEARNED);
                if (!grid_sync(ctl, nblocks, o.timeout_ns)) goto out;
                S.fsz = (long long)read_u64_block(&A->conf_found);
                if (t0) L.confirm_found += S.fsz;
            }
        }
    }
out:
    if (finished && P.samp_feat && s_k >= 0) phase_label(P, s_lo, s_hi, s_k + o.sample_period);
    if (t0) {
        store_state(ctl, S);
        ctl->st_rewrites += L.rewrites;
        ctl->st_nf_marks += L.nf_marks;
        ctl->st_sweeps += L.sweeps;
        ctl->st_visits += L.visits;
        ctl->st_allocs += L.allocs;
        ctl->st_frees += L.frees;
        ctl->st_gc_runs += L.gc_runs;
        ctl->st_confirm += L.confirm;
        ctl->st_confirm_found += L.confirm_found;
        ctl->st_solo_sweeps += L.solo_sweeps;
        ctl->st_refreshes += L.refreshes;
        if (L.frontier_peak > ctl->st_frontier_peak) ctl->st_frontier_peak = L.frontier_peak;
        if (finished) ctl->done = 1;
#ifndef TRS_JIT
        if (cond && (finished || ld_relaxed_s32(&ctl->status) != 0))
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0);
#endif
    }
}

}  // namespace trs
