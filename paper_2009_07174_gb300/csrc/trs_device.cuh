// trs_device.cuh -- device building blocks of the sweep: staged rule tables,
// per-node rule dispatch and rewrite, warp-aggregated allocation and frontier
// pushes, block-scan compaction for garbage collection, and the timed grid
// barrier.  Included by trs_kernels.cu only.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif
#include <stdint.h>

#include "trs_engine.h"

namespace trs {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// memory-model helpers
__device__ __forceinline__ long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s32(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_acqrel_add_u32(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
// Loop-control words are read through L2 (never a stale L1 line).
__device__ __forceinline__ unsigned long long ldcg_u64(const unsigned long long *p) { return __ldcg(p); }
__device__ __forceinline__ long long ldcg_s64(const long long *p) { return __ldcg(p); }

__device__ __forceinline__ int atom_acqrel_add_s32(int *p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void set_status(Ctl *ctl, int st)
{
    atomicCAS(&ctl->status, 0, st);
}

// Grid-wide barrier for co-resident blocks (cooperative launch).  Every wait is
// bounded by timeout_ns; on expiry the status word becomes TRS_ERR_TIMEOUT and
// the barrier returns false, as it does when any block has set an error.
__device__ __noinline__ bool grid_sync(Ctl *ctl, unsigned nblocks, long long timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned gen = ld_relaxed_u32(&ctl->bar_gen);
        __threadfence();
        unsigned arrived = atom_acqrel_add_u32(&ctl->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            red_release_add_u32(&ctl->bar_gen, 1u);
        } else {
            long long t0 = now_ns();
            int spins = 0;
            while (ld_relaxed_u32(&ctl->bar_gen) == gen) {
                // back off once the wait is not short: the waiting blocks'
                // loads all go to the one L2 slice that holds the barrier word
                if (spins >= 64) __nanosleep(spins >= 512 ? 512 : 128);
                if ((++spins & 63) == 0) {
                    if (ld_relaxed_s32(&ctl->status) != 0) { ok = 0; break; }
                    if (now_ns() - t0 > timeout_ns) { set_status(ctl, TRS_ERR_TIMEOUT); ok = 0; break; }
                }
            }
        }
        __threadfence();
        if (ld_relaxed_s32(&ctl->status) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Reference-count change with no result: a relaxed reduction at GPU scope.
// Nothing in a sweep reads the counts back (collection runs between sweeps,
// after the grid barrier's fences), so the change need not return.
__device__ __forceinline__ void red_add_s32(int32_t *p, int32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v));
}
__device__ __forceinline__ void red_or_u32(uint32_t *p, uint32_t v)
{
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v));
}

// ---------------------------------------------------------------------------
// staged rule table
struct Tab {
    const int32_t *w;
    int off_ar, off_first, off_rules;
    __device__ __forceinline__ int arity(int s) const { return w[off_ar + s] & 0xff; }
    __device__ __forceinline__ int first(int s) const { return w[off_first + s]; }
    __device__ __forceinline__ const int32_t *rule(int r) const { return w + off_rules + r * kRuleWords; }
};

__device__ __forceinline__ Tab stage_table(const DevPool &P, int32_t *smem)
{
    for (int t = threadIdx.x; t < P.tab_words; t += blockDim.x) smem[t] = P.tab[t];
    __syncthreads();
    Tab T;
    T.w = smem;
    T.off_ar = smem[4];
    T.off_first = smem[5];
    T.off_rules = smem[6];
    return T;
}

// ---------------------------------------------------------------------------
// per-sweep state, identical in every block
struct State {
    long long k;     // sweep number
    long long n;     // high-water mark at the start of the sweep
    long long fb;    // free ring begin (at sweep start)
    long long fe;    // free ring end
    long long dead;  // reference decrements since the last collection
    long long fsz;   // frontier size
    long long left;  // sweeps left in this call
    long long since; // learned: sweeps since the last refresh
    int cur;         // current frontier buffer
};

// Free-ring positions are kept below 2 * cap by the loop (begin < cap, the ring
// holding at most cap entries), so a ring index is a position less a few
// multiples of cap: no 64-bit division on the allocation path.
__device__ __forceinline__ long long ring_wrap(long long x, long long cap)
{
    while (x >= cap) x -= cap;
    return x;
}

struct Counters {    // per-thread, reduced per block at the end of a phase
    unsigned long long rewrites, nf_marks, visits, allocs, deaths;
};

// A reference count was decremented: mark the slot as a collection
// candidate (one bit, fire and forget) and count a possible death for the
// collection trigger.
__device__ __forceinline__ void mark_candidate(const DevPool &P, int32_t x, Counters &C)
{
    red_or_u32(P.dbm + (x >> 5), 1u << (x & 31));
    C.deaths++;
}



enum { M_PLAIN = 0, M_FRONTIER = 1, M_LEARNED = 2 };
enum { D_SKIP = -1, D_MARK = -2, D_NONE = -3 };

__device__ __forceinline__ bool is_nf_at(int32_t s, long long k) { return s > 0 && s <= k; }

// Readiness of an argument c: R_SWEEP, in normal form as of the start of sweep
// k (the synchronous sweep); R_NOW, in normal form now (an eager learned
// continuation: any positive stamp, read with acquire so that the marker's
// earlier writes are visible).
enum { R_NONE = 0, R_SWEEP = 1, R_NOW = 2 };
__device__ __forceinline__ bool nf_ready(const DevPool &P, int32_t c, long long k, int ready)
{
    return ready == R_NOW ? ld_acquire_s32(&P.nfs[c]) > 0 : is_nf_at(P.nfs[c], k);
}

// A node found to be in normal form in sweep k: plain store, or (learned
// mode) a release store that orders the node's record before the stamp for
// eager continuations that read it with nf_ready(R_NOW).
__device__ __forceinline__ void store_nf(const DevPool &P, int mode, int32_t i, long long k)
{
    if (mode == M_LEARNED) st_release_s32(&P.nfs[i], (int32_t)(k + 1));
    else P.nfs[i] = (int32_t)(k + 1);
}

// Content of a node this lane has just written (head, first arguments and
// parent word), handed to the next step of an eager chain so that it need not
// be read back.
constexpr int kCarryArgs = 4;
struct Carry {
    int32_t h;                  // 0: nothing carried
    int32_t c[kCarryArgs];
    int32_t p;                  // parent word (valid when h != 0)
};

// Prefetch a node record into L1 (a hint: no register, no wait).  Used for
// the records the next step of an eager chain will load.
__device__ __forceinline__ void prefetch_rec(const DevPool &P, int32_t x)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(node_at(P, x)));
}

// Element j of a small per-thread array, by selects (the array stays in
// registers).
template <int N>
__device__ __forceinline__ int32_t pick(const int32_t (&v)[N], int j)
{
    int32_t x = v[0];
#pragma unroll
    for (int t = 1; t < N; t++)
        if (j == t) x = v[t];
    return x;
}

// A node index read where no node need be (an argument word of a node whose
// arity is lower than the pattern assumed): any value is mapped into the
// store, so that the speculative loads below stay in bounds.
__device__ __forceinline__ int32_t in_store(int32_t x, long long cap)
{
    return (uint32_t)x < (uint32_t)cap ? x : 0;
}

constexpr int kPf = 2;  // arguments whose subterms are prefetched

// Readiness and rule dispatch for node i (Sec. 3, derive kernel: a node is
// rewritten when it is live, not in normal form and all its arguments are in
// normal form; the rules of its head are tried in order, Sec. 2).
// Returns a rule slot, D_MARK (no rule matched: normal form) or D_SKIP.
// reg[] receives the nodes matched by the pattern of the returned rule.
//
// Memory-level parallelism: once the arguments are known, the heads of the
// first kPf arguments and the second-level words the head's rules read (the
// table's prefetch plan) are loaded together, and the heads of those
// second-level nodes in one more step, so that a pattern of depth two costs
// two dependent loads instead of one per pattern node and rule.
__device__ __forceinline__ int decide(const DevPool &P, const Tab &T, int32_t i, long long k,
                                      int check_ready, int32_t *reg, int32_t &h_out,
                                      const Carry &cin)
{
    const long long cap = P.cap;
    const bool carried = cin.h != 0;
    // an uncarried node's first two argument words are read with its head
    int32_t h, w0 = 0, w1 = 0;
    if (carried) {
        h = cin.h;
    } else {
        const int4 q = rec_head4(P, i);
        h = q.x;
        w0 = q.y;
        w1 = q.z;
    }
    h_out = h;
    const int aw = T.w[T.off_ar + h];
    const int ar = aw & 0xff, plan = aw >> 8;
    const int r0 = T.first(h), r1 = T.first(h + 1);
    if (!check_ready && r0 == r1) return D_MARK;
    int32_t c[TRS_MAX_ARITY];
#pragma unroll
    for (int j = 0; j < TRS_MAX_ARITY; j++) {
        c[j] = 0;
        if (j < ar)
            c[j] = (carried && j < kCarryArgs) ? cin.c[j]
                   : j == 0                    ? w0
                   : j == 1                    ? w1
                                               : arg_at(P, j, i);
    }
    if (check_ready) {
        bool ready = true;
#pragma unroll
        for (int j = 0; j < TRS_MAX_ARITY; j++)
            if (j < ar && !nf_ready(P, c[j], k, check_ready)) ready = false;
        if (!ready) return D_SKIP;
        if (r0 == r1) return D_MARK;
    }
    int32_t hc[kPf], d0[kPf], d1[kPf], e0[kPf], e1[kPf];
#pragma unroll
    for (int a = 0; a < kPf; a++) {
        hc[a] = d0[a] = d1[a] = e0[a] = e1[a] = 0;
        if (a < ar) {
            if (((plan >> (16 + a)) | (plan >> a) | (plan >> (4 + a))) & 1) {
                // head and first two argument words of the argument together
                const int4 q = rec_head4(P, c[a]);
                hc[a] = q.x;
                d0[a] = q.y;
                d1[a] = q.z;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < kPf; a++) {
        d0[a] = in_store(d0[a], cap);
        d1[a] = in_store(d1[a], cap);
        if ((plan >> (8 + a)) & 1) e0[a] = hs_at(P, d0[a]);
        if ((plan >> (12 + a)) & 1) e1[a] = hs_at(P, d1[a]);
    }
    for (int r = r0; r < r1; r++) {
        const int32_t *R = T.rule(r);
        int npat = R[0] & 0xff;
        const int32_t *pat = T.w + R[2];
        reg[0] = i;
        // argument position of every register that holds one of the first
        // kPf arguments of the redex (15: any other register)
        unsigned long long posw = ~0ull;
        bool ok = true;
        for (int q = 1; q < npat; q++) {
            uint32_t w = (uint32_t)pat[q - 1];
            const int ap = (w >> 8) & 0xff, pr = w & 0xff;
            const int32_t sym = (int32_t)(w >> 16);
            int32_t node, hn = 0;
            bool have = false;
            if (pr == 0) {
                node = pick(c, ap);
                if (ap < kPf) {
                    hn = pick(hc, ap);
                    have = (plan >> (16 + ap)) & 1;
                    posw &= ~(15ull << (4 * q)) | ((unsigned long long)ap << (4 * q));
                }
            } else {
                const int a = (int)((posw >> (4 * pr)) & 15);
                if (a < kPf && ap == 0 && ((plan >> a) & 1)) {
                    node = pick(d0, a);
                    if ((plan >> (8 + a)) & 1) { hn = pick(e0, a); have = true; }
                } else if (a < kPf && ap == 1 && ((plan >> (4 + a)) & 1)) {
                    node = pick(d1, a);
                    if ((plan >> (12 + a)) & 1) { hn = pick(e1, a); have = true; }
                } else {
                    node = arg_at(P, ap, reg[pr]);
                }
            }
            reg[q] = node;
            if (sym != 0) {
                if (!have) hn = hs_at(P, node);
                if (hn != sym) { ok = false; break; }
            }
        }
        if (ok) return r;
    }
    return D_MARK;
}

// Allocation (Sec. 3, get_new_index).  Every new node takes the next position
// of one allocation sequence per sweep: positions below avail = fe - fb name
// the free ring's entries, later ones the fresh slots n, n+1, ... above the
// high-water mark.  A warp claims positions in chunks of kAllocChunk with one
// atomic (warp-uniform state in WarpAlloc) and hands them to its lanes; the
// positions a warp did not use are returned at the end of the phase (fresh
// ones stamped free) and join the ring behind its end.
constexpr int kAllocChunk = 128;

struct WarpAlloc {
    unsigned long long pos, end;  // unused positions [pos, end) of this warp
    unsigned long long chunk;     // claim size (0: exactly what is needed)
    int32_t pre;                  // lane l: the ring slot at position pos + l, else -1
};

// Chunk size for this sweep: all warps' leftovers together stay below half of
// the ring cells this sweep does not read, so returned entries (written behind
// fe during the sweep) never land on a cell that is still to be read; tiny
// stores claim exactly.
__device__ __forceinline__ WarpAlloc warp_alloc_begin(const DevPool &P, const State &S)
{
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long room = (P.cap - (S.fe - S.fb)) / 2;
    long long c = room / (warps > 0 ? warps : 1);
    if (c > kAllocChunk) c = kAllocChunk;
    if (c < 2) c = 0;
    return WarpAlloc{0, 0, (unsigned long long)c, -1};
}

__device__ __forceinline__ int32_t alloc_slot(const DevPool &P, const State &S, unsigned long long pos,
                                              bool &ok)
{
    const long long avail = S.fe - S.fb;
    if ((long long)pos < avail) return P.ring[ring_wrap(S.fb + (long long)pos, P.cap)];
    const long long s = S.n + ((long long)pos - avail);
    if (s >= P.cap) { ok = false; return 0; }
    return (int32_t)s;
}

// Ring entry for position pos of this warp's range, read ahead of its use
// (-1 where the position is a fresh slot or outside the range).
__device__ __forceinline__ int32_t ring_ahead(const DevPool &P, const State &S, unsigned long long pos,
                                              unsigned long long end)
{
    const long long avail = S.fe - S.fb;
    if (pos >= end || (long long)pos >= avail) return -1;
    return P.ring[ring_wrap(S.fb + (long long)pos, P.cap)];
}

// m new slots for each lane (all 32 lanes call).  Lane l keeps the ring entry
// of the warp's l-th next position in a register, loaded after the previous
// allocation, so that ring slots are handed out without waiting for memory.
__device__ __forceinline__ bool warp_alloc(const DevPool &P, const State &S, Acc *A, WarpAlloc &W,
                                           int m, int32_t *out)
{
    const int lane = threadIdx.x & 31;
    int x = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    const int total = __shfl_sync(kFull, x, 31);
    if (total == 0) return true;
    const int excl = x - m;
    const unsigned long long have = W.end - W.pos;
    unsigned long long nb = 0, nsize = 0;
    if ((unsigned long long)total > have) {
        nsize = (unsigned long long)(total - (int)have);
        if (nsize < W.chunk) nsize = W.chunk;
        if (lane == 0) nb = atomicAdd(&A->fl_claims, nsize);
        nb = __shfl_sync(kFull, nb, 0);
    }
    bool ok = true;
    const int mmax = __reduce_max_sync(kFull, m);
#pragma unroll
    for (int j = 0; j < TRS_MAX_RHS; j++) {
        if (j >= mmax) break;
        const unsigned long long q = (unsigned long long)(excl + j);
        const int32_t ahead = __shfl_sync(kFull, W.pre, (int)(q & 31));
        if (j >= m) continue;
        if (q < have && q < 32 && ahead >= 0) {
            out[j] = ahead;
        } else {
            const unsigned long long pos = q < have ? W.pos + q : nb + (q - have);
            out[j] = alloc_slot(P, S, pos, ok);
        }
    }
    if ((unsigned long long)total > have) {
        W.pos = nb + ((unsigned long long)total - have);
        W.end = nb + nsize;
        W.pre = ring_ahead(P, S, W.pos + lane, W.end);
    } else {
        W.pos += (unsigned long long)total;
        const int src = lane + total;
        const int32_t moved = __shfl_sync(kFull, W.pre, src < 32 ? src : 31);
        W.pre = src < 32 ? moved : ring_ahead(P, S, W.pos + lane, W.end);
    }
    if (!ok) set_status(P.ctl, TRS_ERR_POOL_FULL);
    return ok;
}

// End of a phase: give the warp's unused positions back (all 32 lanes call).
__device__ __forceinline__ void warp_alloc_return(const DevPool &P, const State &S, Acc *A,
                                                  WarpAlloc &W)
{
    const int lane = threadIdx.x & 31;
    const long long avail = S.fe - S.fb;
    // positions at or past `limit` would be fresh slots beyond the store:
    // they were never usable and are not given back
    const long long limit = avail + (P.cap - S.n);
    long long cnt = (long long)(W.end - W.pos);
    if ((long long)W.pos + cnt > limit) cnt = limit - (long long)W.pos;
    if (cnt <= 0) { W.pos = W.end; return; }
    unsigned long long rb = 0;
    if (lane == 0) rb = atomicAdd(&A->ret, (unsigned long long)cnt);
    rb = __shfl_sync(kFull, rb, 0);
    for (long long q = lane; q < cnt; q += 32) {
        const unsigned long long pos = W.pos + (unsigned long long)q;
        int32_t slot;
        if ((long long)pos < avail) {
            slot = P.ring[ring_wrap(S.fb + (long long)pos, P.cap)];
        } else {
            slot = (int32_t)(S.n + ((long long)pos - avail));
            P.nfs[slot] = 0;            // never used: a free slot below the new mark
        }
        P.ring[ring_wrap(S.fe + (long long)rb + q, P.cap)] = slot;
    }
    W.pos = W.end;
}

// Warp-aggregated append of cnt entries per lane to a frontier buffer.
__device__ __forceinline__ void warp_push(int32_t *buf, unsigned long long *counter, long long cap,
                                          int cnt, const int32_t *items, Ctl *ctl)
{
    const int lane = threadIdx.x & 31;
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    int total = __shfl_sync(kFull, x, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 31);
    long long at = (long long)base + (x - cnt);
    for (int j = 0; j < cnt; j++) {
        if (at + j < cap) buf[at + j] = items[j];
        else set_status(ctl, TRS_ERR_POOL_FULL);
    }
}

// A node not in normal form has exactly one parent (variables bind only nodes
// in normal form, and uploads are trees); par[] holds it, with the sign bit set
// when the parent's head is unary.  When node i becomes a normal form its
// parent loses one pending argument; the notifier that takes the count to 0
// owns the parent's next visit.  A unary parent has no other argument, so no
// atomic is needed.
__device__ __forceinline__ void notify_parent(const DevPool &P, int32_t pv, int32_t *push, int &npush)
{
    const int32_t p = pv & 0x7fffffff;
    if (p == 0) return;
    if (pv < 0 || atom_acqrel_add_s32(&pend_at(P, p), -1) == 1) {
        push[npush++] = p;
        prefetch_rec(P, p);   // the record the parent's step loads first
    }
}

// Learned frontier: every node enters the next frontier at most once per
// sweep; pend[] holds the number of the sweep it was last queued for.
__device__ __forceinline__ void learned_push(const DevPool &P, int32_t x, long long k_next, int32_t *push,
                                             int &npush)
{
    if (atomicExch(&pend_at(P, x), (int32_t)k_next) != (int32_t)k_next) push[npush++] = x;
}

// Prefetch the records of the first kPf arguments of a continuation of head
// sym that decide() will load (the table's prefetch plan).
__device__ __forceinline__ void prefetch_args(const DevPool &P, const Tab &T, int32_t sym, const Carry &c, int na)
{
    const int plan = T.w[T.off_ar + sym] >> 8;
#pragma unroll
    for (int a = 0; a < kPf; a++)
        if (a < na && a < kCarryArgs && (((plan >> (16 + a)) | (plan >> a) | (plan >> (4 + a))) & 1))
            prefetch_rec(P, c.c[a]);
}

__device__ __forceinline__ int32_t par_word(const Tab &T, int32_t parent, int32_t parent_sym)
{
    return parent | (T.arity(parent_sym) == 1 ? (int32_t)0x80000000 : 0);
}

// Symbol of new node j of a build program (walks the program; j < 16).
__device__ __forceinline__ int32_t build_sym(const int32_t *build, int root_nargs, int j)
{
    int pos = root_nargs;
    for (int t = 0; t < j; t++) pos += 2 + (build[pos] >> 16);
    return build[pos] & 0xffff;
}

// Record that node i is in normal form (no rule matched) in sweep k.
__device__ __forceinline__ void apply_mark(const DevPool &P, int mode, int32_t i, int32_t pv, long long k,
                                           Counters &C, int32_t *push, int &npush)
{
    store_nf(P, mode, i, k);  // in normal form from the next sweep on
    C.nf_marks++;
    if (mode == M_FRONTIER) notify_parent(P, pv, push, npush);
    if (mode == M_LEARNED) {
        const int32_t p = pv & 0x7fffffff;   // the parent may be ready now
        if (p != 0) learned_push(P, p, k + 1, push, npush);
    }
    if (P.act) P.act[i] = min(P.act[i], (int32_t)k);
}

// Apply the decision for node i (rule slot r or D_MARK) in sweep k: rewrite in
// place (Sec. 3, rewrite listing: the redex slot receives the right-hand side's
// root, new nodes receive the other non-variable positions, variables are
// shared; the reference counts of new references are incremented before the
// consumed arguments are decremented) or record that i is in normal form.
// Nodes to visit in the next sweep are appended to push[] (frontier modes).
__device__ __forceinline__ void apply(const DevPool &P, const Tab &T, int mode, int32_t i,
                                      int32_t h, int32_t pv, int r, long long k, const int32_t *reg,
                                      const int32_t *nw, Counters &C, int32_t *push, int &npush,
                                      Carry &last)
{
    const long long cap = P.cap;
    last.h = 0;
    if (r == D_MARK) {
        apply_mark(P, mode, i, pv, k, C, push, npush);
        return;
    }
    const int32_t *R = T.rule(r);
    const int nnew = (R[0] >> 8) & 0xff;
    const int ndelta = (R[0] >> 16) & 0xff;
    const int rootvar = (R[0] >> 24) & 0xff;
    const int32_t *build = T.w + R[3];
    const int32_t *delta = T.w + R[4];
    const int root_nargs = R[5] & 0xff;
    const int root_pend = (R[5] >> 8) & 0xff;
    const int32_t stamp_new = -(int32_t)(k + 1);  // not in normal form, eligible next sweep
    // learned mode queues the nodes a rewrite makes ready for the next sweep,
    // and the one queued last is the eager continuation.  A redex that waits
    // for new arguments is not queued: each of them, on becoming a normal
    // form, queues its parent (one claim per sweep), so the last one can take
    // the redex as its own continuation in the same sweep.

    // new nodes
    int pos = root_nargs;
    for (int j = 0; j < nnew; j++) {
        int32_t w0 = build[pos++];
        int32_t w1 = build[pos++];
        int32_t sym = w0 & 0xffff, na = w0 >> 16;
        int32_t parent = (w1 & 0xffff) - 1, pj = w1 >> 16;
        int32_t x = nw[j];
        hs_at(P, x) = sym;
        Carry cx;
        cx.h = na <= kCarryArgs ? sym : 0;
        cx.p = parent < 0 ? par_word(T, i, R[1]) : par_word(T, nw[parent], build_sym(build, root_nargs, parent));
        for (int a = 0; a < na; a++) {
            int32_t op = build[pos++];
            const int32_t v = (op >> 16) ? nw[op & 0xffff] : reg[op & 0xffff];
            arg_at(P, a, x) = v;
            if (a < kCarryArgs) cx.c[a] = v;
        }
        rc_at(P, x) = 1;
        P.nfs[x] = stamp_new;
        par_at(P, x) = cx.p;
        if (mode == M_LEARNED) {
            // a new node that waits for new arguments is queued (and
            // claimed) by the last of them to become a normal form
            pend_at(P, x) = pj == 0 ? (int32_t)(k + 1) : 0;
            if (pj == 0) {
                push[npush++] = x;
                last = cx;
                prefetch_args(P, T, sym, cx, na);
            }
        } else {
            pend_at(P, x) = pj;
            if (mode == M_FRONTIER && pj == 0) {
                push[npush++] = x;
                last = cx;
                prefetch_args(P, T, sym, cx, na);
            }
        }
    }
    // root that is a variable x: i becomes a copy of x (x is in normal form)
    int32_t xh = 0, xa = 0;
    int32_t xc[TRS_MAX_ARITY];
    if (rootvar) {
        int32_t x = reg[R[1]];
        // the first argument words are read with the head (before the arity
        // is known); words beyond the arity are not used
        const int4 q = rec_head4(P, x);
        xh = q.x;
        xa = T.arity(xh);
        for (int a = 0; a < xa; a++) {
            xc[a] = a < 3 ? quad_word(q, 1 + a) : arg_at(P, a, x);
            red_add_s32(&rc_at(P, xc[a]), 1);
        }
    }
    // net reference changes of matched nodes, positive ones first; fire and
    // forget (no return value on the critical path): a decremented node is
    // marked as a collection candidate, and the collection frees those whose
    // count is then 0
    for (int d = 0; d < ndelta; d++) {
        int32_t w = delta[d];
        int32_t q = w & 0xff, dv = w >> 8;
        red_add_s32(&rc_at(P, reg[q]), dv);
        if (dv < 0) mark_candidate(P, reg[q], C);
    }
    if (rootvar) {
        hs_at(P, i) = xh;
        for (int a = 0; a < xa; a++) arg_at(P, a, i) = xc[a];
        store_nf(P, mode, i, k);
        const int before = npush;
        if (mode == M_FRONTIER) notify_parent(P, pv, push, npush);
        if (mode == M_LEARNED) {
            const int32_t p = pv & 0x7fffffff;
            if (p != 0) learned_push(P, p, k + 1, push, npush);
        }
        if (npush != before) last.h = 0;
    } else {
        hs_at(P, i) = R[1];
        Carry ci;
        ci.h = root_nargs <= kCarryArgs ? R[1] : 0;
        ci.p = pv;  // a rewrite in place keeps the parent
        for (int a = 0; a < root_nargs; a++) {
            int32_t op = build[a];
            const int32_t v = (op >> 16) ? nw[op & 0xffff] : reg[op & 0xffff];
            arg_at(P, a, i) = v;
            if (a < kCarryArgs) ci.c[a] = v;
        }
        if (mode == M_LEARNED) {
            // rewritten: eligible from the next sweep; the release store
            // publishes the record for lanes that read the stamp with acquire
            st_release_s32(&P.nfs[i], -(int32_t)(k + 1));
            // the redex is this lane's: with every argument in normal form it
            // is queued (or continued) without a claim; no argument event can
            // target it (its arguments became normal forms before this step)
            if (root_pend == 0) {
                pend_at(P, i) = (int32_t)(k + 1);
                push[npush++] = i;
                last = ci;
                prefetch_args(P, T, R[1], ci, root_nargs);
            }
        } else {
            pend_at(P, i) = root_pend;
            if (mode == M_FRONTIER && root_pend == 0) {
                push[npush++] = i;
                last = ci;
                prefetch_args(P, T, R[1], ci, root_nargs);
            }
        }
    }
    if (P.act) P.act[i] = min(P.act[i], (int32_t)k);
    C.rewrites++;
    C.allocs += nnew;
}

// Reduce per-thread counters into the sweep accumulator (one atomic per
// counter per block).
__device__ __forceinline__ void flush_counters(Counters &C, Acc *A)
{
    __shared__ unsigned long long s_c[5];
    if (threadIdx.x < 5) s_c[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long v[5] = {C.rewrites, C.nf_marks, C.visits, C.allocs, C.deaths};
#pragma unroll
    for (int t = 0; t < 5; t++) {
        unsigned long long x = v[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_c[t], x);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_c[0]) atomicAdd(&A->rewrites, s_c[0]);
        if (s_c[1]) atomicAdd(&A->nf_marks, s_c[1]);
        if (s_c[2]) atomicAdd(&A->visits, s_c[2]);
        if (s_c[3]) atomicAdd(&A->allocs, s_c[3]);
        if (s_c[4]) atomicAdd(&A->deaths, s_c[4]);
    }
    C = Counters{0, 0, 0, 0, 0};
}

#ifdef TRS_JIT
// Rule matching and rewriting generated for one rule system: the same
// contract as decide() and apply(), with the rules as straight-line code
// (defined by the run-time compiled source after this header).
__device__ __forceinline__ int spec_decide(const DevPool &P, const Tab &T, int32_t i, long long k,
                                           int check_ready, int32_t *reg, int32_t &h_out,
                                           const Carry &cin);
__device__ __forceinline__ void spec_apply(const DevPool &P, const Tab &T, int mode, int32_t i, int32_t h,
                                           int32_t pv, int r, long long k, const int32_t *reg,
                                           const int32_t *nw, Counters &C, int32_t *push, int &npush,
                                           Carry &last);
// new slots a decision needs (its rule's new nodes less the reused slots)
__device__ __forceinline__ int spec_new_count(int d);
#endif

constexpr int kClimb = 64;    // levels of one constructor climb
constexpr int kInPlace = 64;  // steps of one constant chain

// One decision + allocation + application + push for every lane of a warp
// (lane-uniform control flow; `cand` marks lanes with a node to consider).
__device__ __forceinline__ int32_t process_warp(const DevPool &P, const Tab &T, const State &S,
                                                Acc *A, WarpAlloc &W, int mode, bool cand, bool keep,
                                                int32_t i, int check_ready, int32_t *next_buf,
                                                Counters &C, bool eager, Carry &carry, bool climb = false)
{
    int32_t reg[TRS_MAX_PATTERN];
    int32_t nw[TRS_MAX_RHS];
    int32_t push[TRS_MAX_RHS + 2];
    int npush = 0;
    int d = D_NONE;
    int32_t h = 0;
    if (keep) learned_push(P, i, S.k + 1, push, npush);  // learned: not yet eligible, keep it
    // the parent word is loaded together with the node (it is needed when the
    // node turns out to be a normal form), not after the decision
    const int32_t pv = (mode != M_PLAIN && cand) ? (carry.h != 0 ? carry.p : par_at(P, i)) : 0;
    // learned mode with eager continuation: a frontier entry and a lane's
    // claimed continuation can be the same node, so a lane owns a step only
    // once it has swapped the node's stamp from the value it read before
    // deciding to the step's outcome (-(k+1) rewritten, k+1 normal form); the
    // acquire read pairs with the release stamp writes that follow a rewrite
    // or a mark, so the record the decision reads is the one that stamp covers
    const bool own = mode == M_LEARNED && eager && cand;
    int32_t s_seen = 0;
    if (own) {
        s_seen = ld_acquire_s32(&P.nfs[i]);
        if (s_seen > 0 || s_seen == 0 || (check_ready == R_SWEEP && -(long long)s_seen > S.k)) cand = false;
    }
    if (cand) {
        C.visits++;
#ifdef TRS_JIT
        d = spec_decide(P, T, i, S.k, check_ready, reg, h, carry);
#else
        d = decide(P, T, i, S.k, check_ready, reg, h, carry);
#endif
        // learned mode, still waiting: a continuation this lane claimed for
        // the next sweep goes there; an entry is dropped, and the last of its
        // arguments to become a normal form queues it (queueing it here would
        // take the claim that argument needs to continue with it)
        if (mode == M_LEARNED && d == D_SKIP && check_ready == R_NOW) push[npush++] = i;
        if (own && (d >= 0 || d == D_MARK)) {
            const int32_t want = d == D_MARK ? (int32_t)(S.k + 1) : -(int32_t)(S.k + 1);
            if (atomicCAS(&P.nfs[i], s_seen, want) != s_seen) d = D_NONE;  // another lane has it
        }
    }
#ifdef TRS_JIT
    // learned mode with eager continuation allocates every new node: a slot
    // consumed in the middle of a sweep may still be another lane's frontier
    // entry, so it is not reused for a new node in the same sweep
    if (own && d >= 0 && ((d >> 16) & 1)) d = (d & 0xffff) | (((T.rule(d & 0xffff)[0] >> 8) & 0xff) << 17);
    int m = (d >= 0) ? spec_new_count(d) : 0;
#else
    int m = (d >= 0) ? ((T.rule(d)[0] >> 8) & 0xff) : 0;
#endif
    if (__any_sync(kFull, m > 0)) {
        if (!warp_alloc(P, S, A, W, m, nw)) d = D_NONE;
    }
    Carry last;
    last.h = 0;
#ifdef TRS_JIT
    if (d >= 0 || d == D_MARK)
        spec_apply(P, T, mode, i, h, pv, d, S.k, reg, nw, C, push, npush, last);
#else
    if (d >= 0 || d == D_MARK) apply(P, T, mode, i, h, pv, d, S.k, reg, nw, C, push, npush, last);
#endif
    // eager continuation: keep one of the nodes that just became ready (the
    // last pushed: the redex itself, else its parent, else a new node) and
    // process it at once instead of in the next sweep; when this lane wrote
    // that node in this step, its content travels with it
    int32_t cont = -1;
    carry.h = 0;
    if (eager && npush > 0 && (d >= 0 || d == D_MARK)) {
        cont = push[--npush];
        carry = last;
    }
    // Constant chain (frontier mode, eager): when the continuation is node i
    // itself, rewritten in place to a constant (a renaming such as A -> B),
    // the constant's own rule is applied here as long as it needs no new slot.
    // Only constants: chains of rules with arguments (a comparison walking
    // down two numerals) differ in length from lane to lane and would hold a
    // warp's other lanes back.
    if (eager && mode == M_FRONTIER && cont == i && carry.h != 0 && npush == 0 && T.arity(carry.h) == 0 &&
        T.first(carry.h) != T.first(carry.h + 1)) {
        for (int n = 0; n < kInPlace; n++) {
            int32_t h2 = 0;
#ifdef TRS_JIT
            const int d2 = spec_decide(P, T, i, S.k, R_NONE, reg, h2, carry);
            if (d2 < 0 || spec_new_count(d2) > 0) break;
#else
            const int d2 = decide(P, T, i, S.k, R_NONE, reg, h2, carry);
            if (d2 < 0 || ((T.rule(d2)[0] >> 8) & 0xff) > 0) break;
#endif
            Carry last2;
            last2.h = 0;
            C.visits++;
#ifdef TRS_JIT
            spec_apply(P, T, mode, i, h2, pv, d2, S.k, reg, nw, C, push, npush, last2);
#else
            apply(P, T, mode, i, h2, pv, d2, S.k, reg, nw, C, push, npush, last2);
#endif
            cont = -1;
            carry.h = 0;
            if (npush > 0) {
                cont = push[--npush];
                carry = last2;
            }
            if (cont != i || carry.h == 0 || npush != 0 || T.arity(carry.h) != 0 ||
                T.first(carry.h) == T.first(carry.h + 1))
                break;
        }
    }
    // Constructor climb (frontier mode, eager, small frontiers): when node i
    // became a normal form and its unary parent is the continuation, the
    // parent is ready; if its head has no rules it is a normal form too, and so
    // on up the chain.
    // Each level costs one load of the parent's first record words (head,
    // argument, parent word up to arity 2) instead of a step.  The climb stops
    // at a head with rules (handed on as the continuation, its one argument
    // carried), at a binary parent (pending count, as a step would) or after
    // kClimb levels.  Marks and stamps are those the steps would write.
    // Only for solo episodes: with a wide frontier a lane that climbs keeps
    // its warp from taking new entries.
    if (climb && mode == M_FRONTIER && eager && cont >= 0 && carry.h == 0 && (d == D_MARK || d >= 0) &&
        pv < 0 && cont == (pv & 0x7fffffff)) {
        int32_t child = i, p = cont;
        for (int lvl = 0; lvl < kClimb; lvl++) {
            const int4 q = rec_head4(P, p);
            const int32_t ph = q.x;
            if (T.first(ph) != T.first(ph + 1)) {
                cont = p;
                carry.h = ph;
                carry.c[0] = child;
                carry.p = rec_par(rec_ma(P)) < 4 ? quad_word(q, rec_par(rec_ma(P))) : par_at(P, p);
                break;
            }
            P.nfs[p] = (int32_t)(S.k + 1);
            C.nf_marks++;
            const int32_t ppv = rec_ma(P) == 2 ? q.w : par_at(P, p);
            const int32_t pp = ppv & 0x7fffffff;
            cont = -1;
            if (pp == 0) break;
            if (ppv >= 0) {
                if (atom_acqrel_add_s32(&pend_at(P, pp), -1) == 1) cont = pp;
                break;
            }
            child = p;
            p = pp;
            cont = p;
            if (lvl + 1 == kClimb) break;
        }
    }
    if (mode != M_PLAIN && __any_sync(kFull, npush > 0))
        warp_push(next_buf, &A->pushes, P.cap, npush, push, P.ctl);
    return cont;
}

// ---------------------------------------------------------------------------
// phases

// Plain sweep: visit every slot below the high-water mark (Sec. 3, derive
// kernel launched for all n terms).  The stamp array is streamed as int4,
// kPlainUnroll loads per lane in flight (2 KiB per warp) before any of them is
// inspected; slots that are free, in normal form or not yet eligible cost only
// their 4 bytes.
constexpr int kPlainUnroll = 4;

template <int U>
__device__ __forceinline__ void plain_chunks(const DevPool &P, const Tab &T, const State &S, Acc *A,
                                             WarpAlloc &W, Counters &C, long long warp0, long long nwarps)
{
    const int lane = threadIdx.x & 31;
    const long long n = S.n;
    constexpr long long kWarpSlots = 128LL * U;
    const long long nchunks = (n + kWarpSlots - 1) / kWarpSlots;
    for (long long ch = warp0; ch < nchunks; ch += nwarps) {
        // the stamps are reduced to one candidate bit per slot before any
        // candidate is processed, so that only the mask stays live across
        // the rewrite code and the loads are never spilled
        unsigned mask = 0;
        {
            int4 s4[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const long long base = ch * kWarpSlots + (long long)u * 128 + lane * 4;
                if (base + 3 < n) {
                    s4[u] = __ldcs(reinterpret_cast<const int4 *>(P.nfs + base));
                } else {
                    s4[u] = make_int4(0, 0, 0, 0);
                    if (base + 0 < n) s4[u].x = P.nfs[base + 0];
                    if (base + 1 < n) s4[u].y = P.nfs[base + 1];
                    if (base + 2 < n) s4[u].z = P.nfs[base + 2];
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int32_t sv[4] = {s4[u].x, s4[u].y, s4[u].z, s4[u].w};
#pragma unroll
                for (int t = 0; t < 4; t++)
                    if (sv[t] < 0 && -(long long)sv[t] <= S.k) mask |= 1u << (u * 4 + t);
            }
        }
        if (!__any_sync(kFull, mask != 0)) continue;
#pragma unroll 1
        for (int b = 0; b < 4 * U; b++) {
            const bool cand = (mask >> b) & 1;
            if (!__any_sync(kFull, cand)) continue;
            const long long slot = ch * kWarpSlots + (long long)(b >> 2) * 128 + lane * 4 + (b & 3);
            Carry none;
            none.h = 0;
            process_warp(P, T, S, A, W, M_PLAIN, cand, false, (int32_t)slot, R_SWEEP, nullptr, C, false, none);
        }
    }
}

// A small store keeps one int4 load per lane so that its few chunks spread
// over as many warps as possible; a large one keeps kPlainUnroll per lane in
// flight.
__device__ __forceinline__ void phase_plain(const DevPool &P, const Tab &T, const State &S, Acc *A,
                                            long long warp0, long long nwarps)
{
    Counters C{0, 0, 0, 0, 0};
    WarpAlloc W = warp_alloc_begin(P, S);
    if (S.n >= nwarps * 128LL * kPlainUnroll * 2)
        plain_chunks<kPlainUnroll>(P, T, S, A, W, C, warp0, nwarps);
    else
        plain_chunks<1>(P, T, S, A, W, C, warp0, nwarps);
    warp_alloc_return(P, S, A, W);
    flush_counters(C, A);
}

// Frontier sweep: visit the entries of the current frontier buffer.  With an
// eager budget, a lane that makes a node ready keeps processing it (up to
// `eager` nodes per frontier entry), and idle lanes take the next unclaimed
// entries (one atomic per warp), so chains of dependent rewrites advance many
// steps per sweep.  Results and counts are those of the synchronous sweep;
// only the number of sweeps changes.
// `lane_cap`: a warp keeps at most that many lanes busy.  A grid sweep whose
// frontier has fewer entries than the grid has lanes spreads them over all
// warps (about entries / warps per warp) instead of packing 32 chains into
// each of the first warps to claim, which would leave most SMs idle and make
// the packed chains diverge.  With a cap of 1 (no more entries than warps)
// each chain runs on a warp of its own, and the constructor climb (`climb`)
// holds no other lane back.
__device__ __forceinline__ void phase_frontier(const DevPool &P, const Tab &T, const State &S, Acc *A, int mode,
                               long long warp0, long long nwarps, int eager = 0, bool climb = false,
                               int lane_cap = 32)
{
    Counters C{0, 0, 0, 0, 0};
    WarpAlloc W = warp_alloc_begin(P, S);
    const int lane = threadIdx.x & 31;
    const int32_t *cur = P.fq[S.cur];
    int32_t *next = P.fq[S.cur ^ 1];
    if (eager <= 0 || mode == M_PLAIN) {
        const long long nchunks = (S.fsz + 31) / 32;
        for (long long ch = warp0; ch < nchunks; ch += nwarps) {
            long long e = ch * 32 + lane;
            bool cand = false, keep = false;
            int32_t i = 0;
            if (e < S.fsz) {
                i = cur[e];
                int32_t s = P.nfs[i];
                // frontier-mode entries are ready by construction; a learned
                // frontier may hold nodes that are waiting, young or already done
                if (s < 0) {
                    if (-(long long)s <= S.k) cand = true;
                    else keep = (mode == M_LEARNED);
                }
            }
            if (!__any_sync(kFull, cand || keep)) continue;
            Carry none;
            none.h = 0;
            process_warp(P, T, S, A, W, mode, cand, keep, i, mode == M_LEARNED ? R_SWEEP : R_NONE, next, C,
                         false, none);
        }
    } else {
        // learned mode: an entry taken from the frontier is checked against
        // the start of the sweep, like the synchronous sweep (an entry can
        // only be ready if no lane of this sweep made it so, so no two lanes
        // process one node); a continuation this lane claimed is checked
        // against the current state
        int32_t node = -1;
        bool node_fresh = false;
        int steps = 0;
        bool drained = false;
        Carry carry;
        carry.h = 0;
        // stop following chains once this sweep's fresh allocations use half
        // of the slots still above the high-water mark: collection only runs
        // between sweeps
        const unsigned long long claim_budget =
            (unsigned long long)((S.fe - S.fb) + (P.cap - S.n) / 2);
        bool pressure = false;
        int iter = 0;
        // the claim counter is read every 4 steps and its value used 4 steps
        // later, so that the read never stalls the chain
        unsigned long long fl_seen = 0;
        for (;;) {
            if ((++iter & 3) == 0 && !pressure) {
                pressure = __shfl_sync(kFull, fl_seen, 0) > claim_budget;
                if (lane == 0) fl_seen = *(volatile unsigned long long *)&A->fl_claims;
            }
            const bool idle = node < 0;
            const unsigned im0 = __ballot_sync(kFull, idle);
            unsigned im = drained ? 0u : im0;
            if (lane_cap < 32 && im) {
                // the lowest idle lanes, up to the cap on busy lanes
                const int allow = lane_cap - (32 - __popc(im0));
                unsigned r = 0, m = im0;
                for (int t = 0; t < allow && m; t++) {
                    r |= m & (0u - m);
                    m &= m - 1;
                }
                im = r;
            }
            bool fresh_entry = false;
            int32_t kept = -1;   // learned: an entry not yet eligible, queued again
            if (im && !drained) {
                const int leader = __ffs(im) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&A->taken, (unsigned long long)__popc(im));
                base = __shfl_sync(kFull, base, leader);
                if ((long long)base >= S.fsz) drained = true;
                if ((im >> lane) & 1) {
                    long long e = (long long)base + __popc(im & ((1u << lane) - 1u));
                    if (e < S.fsz) {
                        int32_t i = cur[e];
                        int32_t s = P.nfs[i];
                        if (s < 0 && -(long long)s <= S.k) {
                            node = i;
                            fresh_entry = true;
                            carry.h = 0;
                        } else if (s < 0 && mode == M_LEARNED) {
                            kept = i;
                        }
                    }
                }
            }
            if (fresh_entry) {
                steps = 0;
                node_fresh = true;
            }
            const bool cand = node >= 0;
            if (!__any_sync(kFull, cand || kept >= 0)) {
                if (drained) break;
                continue;
            }
            const int ready = mode == M_LEARNED ? (node_fresh ? R_SWEEP : R_NOW) : R_NONE;
            int32_t cont = process_warp(P, T, S, A, W, mode, cand, kept >= 0, cand ? node : (kept >= 0 ? kept : 0),
                                        ready, next, C, true, carry, climb);
            steps++;
            const bool over = cont >= 0 && (steps >= eager || pressure);
            if (__any_sync(kFull, over)) warp_push(next, &A->pushes, P.cap, over ? 1 : 0, &cont, P.ctl);
            node = over ? -1 : cont;
            node_fresh = false;
        }
    }
    warp_alloc_return(P, S, A, W);
    flush_counters(C, A);
}

// Block-wide exclusive scan of a count per thread (warp shuffles, then one
// warp scans the warp totals); returns this thread's offset and writes the
// block total to *total.  Block size <= 1024.
__device__ __forceinline__ int block_scan_count(int v, int *total)
{
    __shared__ int s_w[32];
    __shared__ int s_tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    int in_warp = x - v;
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int v = lane < nw ? s_w[lane] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane < nw) s_w[lane] = x - v;
        if (lane == 31) s_tot = x;
    }
    __syncthreads();
    int off = s_w[wid] + in_warp;
    *total = s_tot;
    __syncthreads();
    return off;
}

// Block-wide exclusive scan of one flag per thread (warp ballot + block scan).
__device__ __forceinline__ int block_scan_flag(bool f, int *total)
{
    return block_scan_count(f ? 1 : 0, total);
}

// Garbage collection (Sec. 3, collect_free_indices).  The paper scans every
// slot for a count of 0.  Here every decrement has set its slot's bit in the
// candidate bitmap, so a collection reads cap / 8 bytes of bitmap instead of
// the store, and visits only the decremented slots:
//   phase_gc_collect: the set bits are cleared and compacted into the
//     candidate list (one atomic per warp and 32 bitmap words);
//   phase_gc_free: each candidate whose count is 0 is claimed by swapping its
//     stamp to 0 (so a slot is freed once even when two threads reach it),
//     releases its arguments and follows the nodes this kills, up to kGcWalk
//     nodes per candidate; dead nodes beyond that get their bit set again and
//     are freed by the next collection.  Freed slots join the free ring with
//     one atomic per warp.
// Warps run independently (no block barrier inside the loops), so a long
// cascade holds back only its own warp.
constexpr int kGcWalk = 24;

__device__ __forceinline__ void phase_gc_collect(const DevPool &P, const State &S, Acc *A,
                                                 long long warp0, long long nwarps)
{
    const int lane = threadIdx.x & 31;
    const long long nwords = (S.n + 31) / 32;
    for (long long g = warp0 * 32; g < nwords; g += nwarps * 32) {
        const long long w = g + lane;
        uint32_t v = 0;
        if (w < nwords) {
            v = P.dbm[w];
            if (v) P.dbm[w] = 0;
            // bits of the last word above the high-water mark belong to no
            // node of this run (a store reused without clearing its bitmap)
            if (w * 32 + 32 > S.n) v &= S.n > w * 32 ? (1u << (S.n - w * 32)) - 1u : 0u;
        }
        const int cnt = __popc(v);
        int x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        const int total = __shfl_sync(kFull, x, 31);
        if (total == 0) continue;
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&A->gc_cand, (unsigned long long)total);
        base = __shfl_sync(kFull, base, 31);
        long long at = (long long)base + (x - cnt);
        while (v) {
            const int bit = __ffs(v) - 1;
            v &= v - 1;
            if (at < P.cap) P.cand[at] = (int32_t)(w * 32 + bit);
            at++;
        }
    }
}

__device__ __forceinline__ void phase_gc_free(const DevPool &P, const Tab &T, const State &S, Acc *A,
                                              long long ncand, long long warp0, long long nwarps)
{
    const int lane = threadIdx.x & 31;
    unsigned long long frees = 0, left = 0;
    if (ncand > P.cap) ncand = P.cap;
    for (long long g = warp0 * 32; g < ncand; g += nwarps * 32) {
        const long long e = g + lane;
        int32_t freed[kGcWalk];
        int nfreed = 0;
        const int32_t x0 = e < ncand ? P.cand[e] : 0;
        // head, arguments and count of the candidate in one go (one sector)
        int4 q0 = make_int4(0, 0, 0, 0);
        int32_t rc0 = 1;
        if (x0 > 0) {
            q0 = rec_head4(P, x0);
            rc0 = rc_at(P, x0);
        }
        if (x0 > 0 && rc0 == 0 && atomicExch(&P.nfs[x0], 0) != 0) {
            int32_t stk[kGcWalk];
            int sp = 0;
            stk[sp++] = x0;
            while (sp > 0) {
                const int32_t x = stk[--sp];
                freed[nfreed++] = x;
                const int4 q = x == x0 ? q0 : rec_head4(P, x);
                const int ar = T.arity(q.x);
                // the first two decrements are in flight together
                int od[2];
#pragma unroll
                for (int a = 0; a < 2; a++) od[a] = a < ar ? atomicSub(&rc_at(P, quad_word(q, 1 + a)), 1) : 0;
                for (int a = 0; a < ar; a++) {
                    const int32_t c = a < 3 ? quad_word(q, 1 + a) : arg_at(P, a, x);
                    const int old = a < 2 ? (a == 0 ? od[0] : od[1]) : atomicSub(&rc_at(P, c), 1);
                    if (old != 1) continue;
                    if (nfreed + sp < kGcWalk) {
                        if (atomicExch(&P.nfs[c], 0) != 0) stk[sp++] = c;
                    } else {
                        red_or_u32(P.dbm + (c >> 5), 1u << (c & 31));  // freed by the next collection
                        left++;
                    }
                }
            }
        }
        frees += nfreed;
        // warp-aggregated append of the freed slots to the ring
        int x = nfreed;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        const int total = __shfl_sync(kFull, x, 31);
        if (total == 0) continue;
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&A->gc_append, (unsigned long long)total);
        base = __shfl_sync(kFull, base, 31);
        long long r = ring_wrap(S.fe + (long long)base + (x - nfreed), P.cap);
        for (int j = 0; j < nfreed; j++) {
            P.ring[r] = freed[j];
            if (++r == P.cap) r = 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        frees += __shfl_down_sync(kFull, frees, o);
        left += __shfl_down_sync(kFull, left, o);
    }
    if (lane == 0) {
        if (frees) atomicAdd(&A->gc_frees, frees);
        if (left) atomicAdd(&A->gc_deaths, left);
    }
}

// Seed / confirmation scan (frontier mode): recompute, for every live node not
// in normal form, how many arguments are not in normal form, and append the
// nodes with none to the current frontier buffer.  Run at the start of a
// normalisation and, as the full confirmation sweep, whenever the frontier
// becomes empty.
__device__ __forceinline__ void phase_seed(const DevPool &P, const Tab &T, const State &S, Acc *A,
                                           long long block0, long long nblocks, int mode = M_FRONTIER)
{
    __shared__ unsigned long long s_base;
    int32_t *buf = P.fq[S.cur];
    const long long n = S.n;
    const long long per = (long long)blockDim.x * 4;
    const long long nchunks = (n + per - 1) / per;
    for (long long ch = block0; ch < nchunks; ch += nblocks) {
        const long long base = ch * per + (long long)threadIdx.x * 4;
        int32_t sv[4] = {0, 0, 0, 0};
        if (base + 4 <= n) {
            const int4 s4 = *reinterpret_cast<const int4 *>(P.nfs + base);
            sv[0] = s4.x; sv[1] = s4.y; sv[2] = s4.z; sv[3] = s4.w;
        } else {
            for (int t = 0; t < 4; t++)
                if (base + t < n) sv[t] = P.nfs[base + t];
        }
        int32_t ready[4];
        int nready = 0;
        for (int t = 0; t < 4; t++) {
            const long long i = base + t;
            if (i < 1 || sv[t] >= 0) continue;
            const int ar = T.arity(hs_at(P, i));
            int cnt = 0;
            for (int a = 0; a < ar; a++) {
                const int32_t c = arg_at(P, a, i);
                if (!is_nf_at(P.nfs[c], S.k)) cnt++;
            }
            const bool rdy = cnt == 0 && -(long long)sv[t] <= S.k;
            // frontier mode: pending-argument count; learned mode: the queue
            // tag of the sweep the ready nodes join
            if (mode != M_LEARNED) pend_at(P, i) = cnt;
            else if (rdy) pend_at(P, i) = (int32_t)S.k;
            if (rdy) ready[nready++] = (int32_t)i;
        }
        // a chunk without ready nodes (every chunk of a confirmation scan
        // that finds nothing) costs one barrier instead of a block scan
        if (!__syncthreads_or(nready > 0)) continue;
        int total = 0;
        const int off = block_scan_count(nready, &total);
        if (total > 0) {
            if (threadIdx.x == 0) s_base = atomicAdd(&A->conf_found, (unsigned long long)total);
            __syncthreads();
            for (int j = 0; j < nready; j++)
                if ((long long)s_base + off + j < P.cap) buf[s_base + off + j] = ready[j];
            __syncthreads();
        }
    }
}

}  // namespace trs

#include "trs_mlp.cuh"

namespace trs {

// Local view of node i for the predictor: its head, its arguments' heads (0
// beyond the head's arity) and which arguments are in normal form at sweep k.
__device__ __forceinline__ void node_features(const DevPool &P, const Tab &T, int32_t i, long long k,
                                              int &h, int32_t *a, unsigned &bits)
{
    h = hs_at(P, i);
    const int ar = T.arity(h);
    bits = 0;
#pragma unroll
    for (int j = 0; j < TRS_MAX_ARITY; j++) {
        a[j] = 0;
        if (j < P.ma && j < ar) {
            const int32_t c = arg_at(P, j, i);
            a[j] = hs_at(P, c);
            if (is_nf_at(P.nfs[c], k)) bits |= 1u << j;
        }
    }
}

// Learned-frontier refresh: score every live node that is not in normal form
// with the predictor (BF16 weights in shared memory, FP32 accumulation) and
// append those at or above the threshold, not queued already, to the current
// frontier buffer.
// Counts all such nodes too: a refresh that finds none is the full sweep that
// confirms termination.
__device__ __forceinline__ void phase_refresh(const DevPool &P, const Tab &T, const MlpView &M, const State &S, Acc *A,
                              float thr, long long block0, long long nblocks)
{
    __shared__ unsigned long long s_base;
    int32_t *buf = P.fq[S.cur];
    const long long n = S.n;
    const long long per = (long long)blockDim.x;
    const long long nchunks = (n + per - 1) / per;
    unsigned long long pend = 0;
    for (long long ch = block0; ch < nchunks; ch += nblocks) {
        const long long i = ch * per + threadIdx.x;
        const bool pending = i >= 1 && i < n && P.nfs[i] < 0;
        int h = 0;
        int32_t a[TRS_MAX_ARITY];
        unsigned bits = 0;
        if (pending) node_features(P, T, (int32_t)i, S.k, h, a, bits);
        else {
#pragma unroll
            for (int j = 0; j < TRS_MAX_ARITY; j++) a[j] = 0;
        }
        const float p = mlp_warp_prob(M, pending, h, a, bits);
        // the selection joins the entries the last sweep queued (those carry
        // this sweep's number in their pending word)
        const bool sel = pending && p >= thr && pend_at(P, i) != (int32_t)S.k;
        if (sel) pend_at(P, i) = (int32_t)S.k;
        pend += pending ? 1 : 0;
        int total = 0;
        const int off = block_scan_flag(sel, &total);
        if (total > 0) {
            if (threadIdx.x == 0) s_base = atomicAdd(&A->refresh_sel, (unsigned long long)total);
            __syncthreads();
            const long long at = S.fsz + (long long)s_base + off;
            if (sel && at < P.cap) buf[at] = (int32_t)i;
            __syncthreads();
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pend += __shfl_down_sync(kFull, pend, o);
    if ((threadIdx.x & 31) == 0 && pend) atomicAdd(&A->pending, pend);
}

// Predictor traces, labels: row r was sampled at sweep s; its node acted
// (was rewritten or marked) before sweep k_until iff act[slot] < k_until.
__device__ __forceinline__ void phase_label(const DevPool &P, long long lo, long long hi, long long k_until)
{
    for (long long r = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; r < hi;
         r += (long long)gridDim.x * blockDim.x)
        P.samp_label[r] = (long long)P.act[P.samp_slot[r]] < k_until ? 1.f : 0.f;
}

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    // integer finaliser (xorshift-multiply), used only to pick sample nodes
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Predictor traces, samples: a hashed subset of the live nodes not in normal
// form at the start of sweep k; their features become rows and their act[]
// entries restart.
__device__ __forceinline__ void phase_sample(const DevPool &P, const Tab &T, const State &S, const LaunchOpts &o)
{
    __shared__ unsigned long long s_base;
    const long long n = S.n;
    const long long per = (long long)blockDim.x;
    const long long nchunks = (n + per - 1) / per;
    const int F = 2 + P.ma;
    for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long long i = ch * per + threadIdx.x;
        bool take = false;
        if (i >= 1 && i < n) {
            const int32_t s = P.nfs[i];
            if (s < 0 && -(long long)s <= S.k)
                take = mix32((uint32_t)i * 0x9E3779B1u ^ (uint32_t)S.k * 0x85EBCA77u ^ o.sample_seed) <
                       o.sample_thresh;
        }
        int total = 0;
        const int off = block_scan_flag(take, &total);
        if (total > 0) {
            if (threadIdx.x == 0) s_base = atomicAdd((unsigned long long *)&P.ctl->samp_n, (unsigned long long)total);
            __syncthreads();
            const long long r = (long long)s_base + off;
            if (take && r < P.samp_cap) {
                int h;
                int32_t a[TRS_MAX_ARITY];
                unsigned bits;
                node_features(P, T, (int32_t)i, S.k, h, a, bits);
                int32_t *row = P.samp_feat + r * F;
                row[0] = h;
                for (int j = 0; j < P.ma; j++) row[1 + j] = a[j];
                row[1 + P.ma] = (int32_t)bits;
                P.samp_slot[r] = (int32_t)i;
                P.act[i] = 0x7fffffff;
            }
            __syncthreads();
        }
    }
}

}  // namespace trs
