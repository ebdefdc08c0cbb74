// trs_transfer.cu -- terms between host and device without host-side tree
// work: term_upload_batch builds the node records of a batch on the device
// from the preorder symbols, and term_download_batch writes the canonical
// serialisation of large stores on the device, so that only preorder symbols
// and offsets cross the link in either direction.
//
// Upload.  With a[i] the arity of the i-th symbol of the concatenated batch,
// e[i] = 1 + sum_{j<i} (a[j] - 1) counts the argument places still open
// before symbol i is placed (a preorder fills the most recently opened place
// first, Sec. 2 terms).  The parent of symbol i is the last j < i with
// e[j] <= e[i] (every node of the previous sibling's subtree has a larger e),
// and i is its argument a[j] - 1 - (e[i] - e[j]); a term's root has no such
// j.  This previous-smaller-or-equal search runs as one sequential stack per
// thread over a chunk of 256 symbols; a sparse table of chunk minima then
// finds the chunk of every symbol whose parent lies before its own chunk.
// The batch is validated on the device (symbols in range, term t starting at
// e = 1 - t, exactly one parentless symbol per term) before any record is
// written.
//
// Download.  A normal form is a DAG (variables are shared, Sec. 3), so the
// unfolded tree of a root can be far larger than the nodes it occupies, and a
// single root can be huge (one term of millions of nodes).  The pass works on
// "items": a preorder sequence in which each entry is either a symbol already
// placed (stored as -symbol) or a reference to a subtree still to be written
// (stored as its node index).  It starts from the roots and, for a bounded
// number of rounds, replaces every reference by its head symbol followed by
// references to its arguments (a count, a scan for positions, a write), so
// that the top of each tree is unfolded breadth-first into many independent
// subtrees.  Then one thread per item counts its subtree (depth-first, a small
// stack), a scan turns the counts into output offsets, and one thread per item
// writes its subtree's preorder at its offset.  Output larger than the staging
// area is written in windows.
//
// Every loop is bounded and every index is checked against the high-water
// mark and the signature: a corrupt store or a stack that would overflow sets
// a status word instead of faulting.
#include <cuda_runtime.h>

#include <stdint.h>

#include <vector>

#include "trs_engine.h"

namespace trs {

namespace dl {

constexpr int kStack = 64;   // depth-first stack per thread (right siblings pending)
constexpr int kScanBlocks = 608;
constexpr int kThreads = 256;

struct Ctl {
    long long n_items;    // items of the current buffer
    long long total;      // scratch: total after a count + scan
    int cur;              // current item buffer
    int stopped;          // expansion has stopped
    int status;           // 0, TRS_ERR_STATE (corrupt store / dead root) or
                          // TRS_ERR_TOO_BIG (a depth-first stack would overflow)
    int overflow;         // the chunk pool ran out: emission walks the store again
    unsigned long long chunk_next;  // chunks handed out
};

// The counting walk also keeps the symbols it visits, in chunks of kCh words
// from a pool (word 0: the next chunk of the same item, or -1), so that the
// emission copies them instead of walking the store a second time.
constexpr int kCh = 64;

__device__ __forceinline__ void fail(Ctl *c, int st) { atomicCAS(&c->status, 0, st); }

__device__ __forceinline__ long long clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// A walk gives up (TRS_ERR_TIMEOUT) after limit_ns: only a corrupt store
// (a cycle) could make it run that long.

__device__ __forceinline__ int arity_of(const int32_t *tab, int32_t s) { return tab[tab[4] + s] & 0xff; }

// A node index is usable if it lies in [1, n_top) and its head is a symbol.
__device__ __forceinline__ bool node_ok(const DevPool &P, long long n_top, int32_t x, int32_t &h)
{
    if (x < 1 || (long long)x >= n_top) return false;
    h = P.rec[(long long)x * P.rs + kRecHead];
    return h >= 1 && h < P.nsym;
}

// Roots: in range, not free (stamp != 0) and referenced (count > 0).
__global__ void k_roots(DevPool P, long long n_top, const int32_t *roots, int nroots, int32_t *items,
                        int32_t *starts, Ctl *c)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nroots; r += gridDim.x * blockDim.x) {
        const int32_t x = roots[r];
        int32_t h = 0;
        if (!node_ok(P, n_top, x, h) || P.nfs[x] == 0 || P.rec[(long long)x * P.rs + rec_rc(P.ma)] <= 0)
            fail(c, TRS_ERR_STATE);
        items[r] = x;
        starts[r] = r;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        starts[nroots] = nroots;
        c->n_items = nroots;
        c->cur = 0;
        c->stopped = 0;
    }
}

// Expansion round, step 1: output count of every item (1 for a symbol or a
// leaf, 1 + arity for an inner node).
__global__ void k_expand_count(DevPool P, long long n_top, int32_t *const *items, long long *cnt, Ctl *c)
{
    if (c->stopped || c->status) return;
    const int32_t *it = items[c->cur];
    const long long n = c->n_items;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int32_t x = it[e];
        long long k = 1;
        if (x > 0) {
            int32_t h = 0;
            if (!node_ok(P, n_top, x, h)) fail(c, TRS_ERR_STATE);
            else k = 1 + arity_of(P.tab, h);
        }
        cnt[e] = k;
    }
}

// Expansion round, step 3 (after the scan): write the expanded items if they
// fit, else stop expanding (the current items stay).
__global__ void k_expand_write(DevPool P, int32_t *const *items, int32_t *const *starts, const long long *off,
                               long long cap_items, int nroots, Ctl *c)
{
    if (c->stopped || c->status) return;
    const long long total = c->total;
    const long long n = c->n_items;
    if (total > cap_items || total == n) return;  // no room, or nothing left to unfold
    const int32_t *it = items[c->cur];
    int32_t *out = items[c->cur ^ 1];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int32_t x = it[e];
        long long o = off[e];
        if (x <= 0) {
            out[o] = x;
            continue;
        }
        const int32_t *r = P.rec + (long long)x * P.rs;
        const int32_t h = r[kRecHead];
        out[o++] = -h;
        const int a = arity_of(P.tab, h);
        for (int j = 0; j < a; j++) out[o++] = r[rec_arg(j)];
    }
    const int32_t *st = starts[c->cur];
    int32_t *st2 = starts[c->cur ^ 1];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= nroots; r += (long long)gridDim.x * blockDim.x)
        st2[r] = r == nroots ? (int32_t)total : (int32_t)off[st[r]];
}

// Last block of a round: make the written buffer current.
__global__ void k_expand_flip(Ctl *c, long long cap_items)
{
    if (c->stopped || c->status) return;
    if (c->total > cap_items || c->total == c->n_items) {
        c->stopped = 1;
        return;
    }
    c->n_items = c->total;
    c->cur ^= 1;
}

// Size of every item: 1 for a symbol, the unfolded subtree for a reference
// (depth first; the stack holds the pending right siblings).
// Read-ahead: a chain built by rewriting usually lies in consecutive slots
// (the rewrites reuse the slots of the numeral they consume in order, or take
// consecutive fresh slots), so whenever the walk has to load a record it
// loads the first words of the kAhead records from that slot on together,
// and a node whose slot is among them costs no load of its own.
constexpr int kAhead = 8;

__global__ void k_sizes(DevPool P, long long n_top, int32_t *const *items, long long *sz, Ctl *c,
                        long long limit_ns, int32_t *chunks, long long chunk_cap, int32_t *ihead)
{
    const int32_t *it = items[c->cur];
    const long long n = c->n_items;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int32_t x0 = it[e];
        if (x0 <= 0) {
            sz[e] = 1;
            ihead[e] = -1;
            continue;
        }
        int32_t stk[kStack];
        int sp = 0;
        long long cntv = 0;
        int32_t x = x0;
        int32_t head = -1, chk = -1;
        int fill = kCh;
        bool keep = true;
        const long long t0 = clock_ns();
        long long base = -kAhead - 1;   // slots base .. base + kAhead - 1 are in ahead[]
        int4 ahead[kAhead];
        for (;;) {
            if (x < 1 || (long long)x >= n_top) { fail(c, TRS_ERR_STATE); break; }
            if ((long long)x < base || (long long)x >= base + kAhead) {
                base = x;
#pragma unroll
                for (int j = 0; j < kAhead; j++) {
                    const long long y = base + j < n_top ? base + j : base;
                    ahead[j] = *reinterpret_cast<const int4 *>(P.rec + y * P.rs);
                }
            }
            int4 q = ahead[0];
#pragma unroll
            for (int j = 1; j < kAhead; j++)
                if ((long long)x - base == j) q = ahead[j];
            const int32_t h = q.x;
            if (h < 1 || h >= P.nsym) { fail(c, TRS_ERR_STATE); break; }
            cntv++;
            if (keep) {
                if (fill == kCh) {
                    const unsigned long long nc = atomicAdd(&c->chunk_next, 1ull);
                    if ((long long)nc >= chunk_cap) {
                        keep = false;
                        c->overflow = 1;
                    } else {
                        if (chk >= 0) chunks[(long long)chk * kCh] = (int32_t)nc;
                        else head = (int32_t)nc;
                        chk = (int32_t)nc;
                        chunks[(long long)chk * kCh] = -1;
                        fill = 1;
                    }
                }
                if (keep) chunks[(long long)chk * kCh + fill++] = h;
            }
            if ((cntv & 4095) == 0 && (clock_ns() - t0 > limit_ns || c->status)) {
                fail(c, TRS_ERR_TIMEOUT);
                break;
            }
            const int32_t *r = P.rec + (long long)x * P.rs;
            const int a = arity_of(P.tab, h);
            if (a > 0) {
                if (sp + a - 1 > kStack) { fail(c, TRS_ERR_TOO_BIG); break; }
                for (int j = a - 1; j >= 1; j--) stk[sp++] = j == 1 ? q.z : j == 2 ? q.w : r[rec_arg(j)];
                x = q.y;
            } else {
                if (sp == 0) break;
                x = stk[--sp];
            }
        }
        sz[e] = cntv;
        ihead[e] = head;
    }
}

// Emission from the kept chunks: the items whose output range meets [lo, hi).
// One warp takes 32 items: their lanes write the placed symbols, then the
// warp copies each subtree item's chunks in turn, one chunk per step (lane l
// moves symbols l + 1 and l + 33 of the chunk, coalesced), so that a long item
// costs one dependent load (the next-chunk word) per 63 symbols.
__global__ void k_copy(int32_t *const *items, const long long *off, const int32_t *ihead, const int32_t *chunks,
                       int32_t *out, long long lo, long long hi, Ctl *c)
{
    if (c->status) return;
    const unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t *it = items[c->cur];
    const long long n = c->n_items;
    const long long warp0 = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long g = warp0 * 32; g < n; g += nwarps * 32) {
        const long long el = g + lane;
        bool ref = false;
        if (el < n) {
            const long long pos = off[el];
            const long long end = off[el + 1];
            if (end > lo && pos < hi) {
                const int32_t x0 = it[el];
                if (x0 <= 0) out[pos - lo] = -x0;
                else ref = true;
            }
        }
        unsigned todo = __ballot_sync(kAll, ref);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const long long e = g + src;
            const long long end = off[e + 1];
            long long base = off[e];   // output position of the current chunk's first symbol
            long long ch = ihead[e];
            while (ch >= 0 && base < end && base < hi) {
                if (base + (kCh - 1) > lo) {
#pragma unroll
                    for (int pass = 0; pass < 2; pass++) {
                        const int k = 1 + lane + 32 * pass;
                        const long long p = base + (k - 1);
                        if (k < kCh && p < end && p >= lo && p < hi) out[p - lo] = chunks[ch * kCh + k];
                    }
                }
                ch = chunks[ch * kCh];
                base += kCh - 1;
            }
        }
    }
}

// Write the preorder of every item whose output range meets [lo, hi) into
// out[0 .. hi - lo).
__global__ void k_emit(DevPool P, long long n_top, int32_t *const *items, const long long *off, int32_t *out,
                       long long lo, long long hi, Ctl *c)
{
    if (c->status) return;
    const int32_t *it = items[c->cur];
    const long long n = c->n_items;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        long long pos = off[e];
        const long long end = off[e + 1];
        if (end <= lo || pos >= hi) continue;
        const int32_t x0 = it[e];
        if (x0 <= 0) {
            out[pos - lo] = -x0;
            continue;
        }
        int32_t stk[kStack];
        int sp = 0;
        int32_t x = x0;
        while (pos < hi) {
            int32_t h = 0;
            if (!node_ok(P, n_top, x, h)) { fail(c, TRS_ERR_STATE); break; }
            if (pos >= lo) out[pos - lo] = h;
            pos++;
            const int32_t *r = P.rec + (long long)x * P.rs;
            const int a = arity_of(P.tab, h);
            if (a > 0) {
                if (sp + a - 1 > kStack) { fail(c, TRS_ERR_TOO_BIG); break; }
                for (int j = a - 1; j >= 1; j--) stk[sp++] = r[rec_arg(j)];
                x = r[rec_arg(0)];
            } else {
                if (sp == 0) break;
                x = stk[--sp];
            }
        }
    }
}

// Per-root output offsets from the item offsets.
__global__ void k_root_offsets(int32_t *const *starts, const long long *off, int nroots, long long *roff, Ctl *c)
{
    const int32_t *st = starts[c->cur];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r <= nroots; r += gridDim.x * blockDim.x)
        roff[r] = off[st[r]];
}

// ---------------------------------------------------------------------------
// Exclusive scan of n int64 values in place (v[n] receives the total, and
// c->total too).  Three launches: per-block sums over contiguous chunks, a
// scan of the block sums by one block, and a per-block rescan with the
// block's offset.
__device__ __forceinline__ long long block_excl_scan(long long x, long long *s_w, long long &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
    }
    if (lane == 31) s_w[wid] = y;
    __syncthreads();
    if (wid == 0) {
        long long v = lane < nw ? s_w[lane] : 0;
        long long z = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += t;
        }
        if (lane < nw) s_w[lane] = z - v;
        if (lane == 31) s_w[32] = z;
    }
    __syncthreads();
    const long long r = y - x + s_w[wid];
    total = s_w[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void chunk_of(long long n, long long &b, long long &e)
{
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    b = per * blockIdx.x;
    e = b + per < n ? b + per : n;
    if (b > n) b = n;
}

// mode 0: n = n_fixed; 1: the items of an expansion round (nothing once the
// expansion has stopped); 2: the current items
__device__ __forceinline__ bool scan_skip(const Ctl *c, int mode) { return c->status || (mode == 1 && c->stopped); }
__device__ __forceinline__ long long scan_n(const Ctl *c, int mode, long long n_fixed)
{
    return mode == 0 ? n_fixed : c->n_items;
}

__global__ void k_scan_sums(const long long *v, const Ctl *c, long long *bsum, int mode, long long n_fixed)
{
    if (scan_skip(c, mode)) return;
    const long long n = scan_n(c, mode, n_fixed);
    long long b, e;
    chunk_of(n, b, e);
    long long s = 0;
    for (long long i = b + threadIdx.x; i < e; i += blockDim.x) s += v[i];
    __shared__ long long s_w[33];
    long long tot;
    block_excl_scan(s, s_w, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_top(long long *bsum, int nb, Ctl *c, int mode)
{
    if (scan_skip(c, mode)) return;
    __shared__ long long s_w[33];
    long long run = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long x = i < nb ? bsum[i] : 0;
        long long tot;
        const long long ex = block_excl_scan(x, s_w, tot);
        if (i < nb) bsum[i] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) {
        bsum[nb] = run;
        c->total = run;
    }
}

__global__ void k_scan_apply(long long *v, const long long *bsum, Ctl *c, int mode, long long n_fixed)
{
    if (scan_skip(c, mode)) return;
    const long long n = scan_n(c, mode, n_fixed);
    long long b, e;
    chunk_of(n, b, e);
    __shared__ long long s_w[33];
    long long run = bsum[blockIdx.x];
    for (long long base = b; base < e; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const long long x = i < e ? v[i] : 0;
        long long tot;
        const long long ex = block_excl_scan(x, s_w, tot);
        if (i < e) v[i] = run + ex;
        run += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) v[n] = bsum[gridDim.x];
}

}  // namespace dl

// ---------------------------------------------------------------------------
// Upload kernels
namespace up {

constexpr int kChunk = 256;   // symbols per thread in the chunk-local stack pass
constexpr int kThreads = 256;
constexpr int kScanBlocks = 608;

struct Ctl {
    int status;           // 0 or TRS_ERR_BAD_TERM
    int pad;
    long long parentless; // symbols without a parent (must be one per term)
};

__device__ __forceinline__ void fail(Ctl *c) { atomicCAS(&c->status, 0, (int)TRS_ERR_BAD_TERM); }
__device__ __forceinline__ int arity_of(const int32_t *tab, int32_t s) { return tab[tab[4] + s] & 0xff; }

__device__ __forceinline__ void chunk_range(long long n, long long &b, long long &e)
{
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    b = per * blockIdx.x;
    e = b + per < n ? b + per : n;
    if (b > n) b = n;
}

// a[i] - 1 of a symbol (an out-of-range symbol fails the batch and counts 0)
__device__ __forceinline__ long long step_of(const int32_t *tab, int nsym, int32_t sym, Ctl *c)
{
    if (sym < 1 || sym >= nsym) {
        fail(c);
        return 0;
    }
    return (long long)arity_of(tab, sym) - 1;
}

__global__ void k_sums(const int32_t *flat, long long n, const int32_t *tab, int nsym, long long *bsum, Ctl *c)
{
    long long b, e;
    chunk_range(n, b, e);
    long long sum = 0;
    for (long long i = b + threadIdx.x; i < e; i += blockDim.x) sum += step_of(tab, nsym, flat[i], c);
    __shared__ long long s_w[33];
    long long tot;
    dl::block_excl_scan(sum, s_w, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_top(long long *bsum, int nb)
{
    __shared__ long long s_w[33];
    long long run = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long x = i < nb ? bsum[i] : 0;
        long long tot;
        const long long ex = dl::block_excl_scan(x, s_w, tot);
        if (i < nb) bsum[i] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) bsum[nb] = run;
}

// e[i] = 1 + exclusive prefix of (a - 1); a valid batch keeps e in
// [1 - nterms, n] (open places never exceed the symbols still to come)
__global__ void k_open(const int32_t *flat, long long n, long long nterms, const int32_t *tab, int nsym,
                       const long long *bsum, int32_t *e_out, Ctl *c)
{
    long long b, e;
    chunk_range(n, b, e);
    __shared__ long long s_w[33];
    long long run = bsum[blockIdx.x];
    for (long long base = b; base < e; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const long long x = i < e ? step_of(tab, nsym, flat[i], c) : 0;
        long long tot;
        const long long ex = dl::block_excl_scan(x, s_w, tot);
        if (i < e) {
            const long long v = 1 + run + ex;
            if (v < 1 - nterms || v > n) fail(c);
            e_out[i] = (int32_t)(v < -(1LL << 30) ? -(1LL << 30) : v > (1LL << 30) ? (1LL << 30) : v);
        }
        run += tot;
    }
}

// Chunk-local previous-smaller-or-equal: one thread per chunk, a stack of
// chunk positions; -1 where the answer lies before the chunk.  Also the
// chunk minimum.
__global__ void k_local(const int32_t *e, long long n, int32_t *par, int32_t *cmin)
{
    const long long nch = (n + kChunk - 1) / kChunk;
    for (long long ch = blockIdx.x * (long long)blockDim.x + threadIdx.x; ch < nch;
         ch += (long long)gridDim.x * blockDim.x) {
        const long long lo = ch * kChunk;
        const long long hi = lo + kChunk < n ? lo + kChunk : n;
        unsigned char stk[kChunk];
        int sp = 0;
        int32_t mn = 0x7fffffff;
        for (long long i = lo; i < hi; i++) {
            const int32_t v = e[i];
            while (sp > 0 && e[lo + stk[sp - 1]] > v) sp--;
            par[i] = sp > 0 ? (int32_t)(lo + stk[sp - 1]) : -1;
            stk[sp++] = (unsigned char)(i - lo);
            if (v < mn) mn = v;
        }
        cmin[ch] = mn;
    }
}

// Sparse table level k from level k - 1: minimum over 2^k chunks.
__global__ void k_table(int32_t *st, long long nch, int k)
{
    const int32_t *prev = st + (long long)(k - 1) * nch;
    int32_t *cur = st + (long long)k * nch;
    const long long half = 1LL << (k - 1);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nch; c += (long long)gridDim.x * blockDim.x)
        cur[c] = c + half < nch ? min(prev[c], prev[c + half]) : prev[c];
}

// Symbols whose parent lies before their chunk: the nearest earlier chunk
// with a minimum <= e[i] (greedy descent over the sparse table), then, from
// that chunk's last symbol, the chain of previous-smaller-or-equal links
// down to the first symbol <= e[i].  Symbols with none are term roots.
__global__ void k_resolve(const int32_t *e, long long n, int32_t *par, const int32_t *st, long long nch,
                          int levels, Ctl *c)
{
    unsigned long long roots = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (par[i] >= 0) continue;
        const int32_t v = e[i];
        long long pos = i / kChunk - 1;
        for (int k = levels - 1; k >= 0; k--) {
            const long long span = 1LL << k;
            if (pos - span + 1 >= 0 && st[(long long)k * nch + pos - span + 1] > v) pos -= span;
        }
        if (pos < 0) {
            roots++;
            continue;
        }
        const long long lo = pos * kChunk;
        long long j = lo + kChunk - 1 < n - 1 ? lo + kChunk - 1 : n - 1;
        int guard = 0;
        while (e[j] > v) {
            const int32_t nx = par[j];
            if (nx < lo || nx >= j || ++guard > kChunk) {
                fail(c);
                j = -1;
                break;
            }
            j = nx;
        }
        if (j >= 0) par[i] = (int32_t)j;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) roots += __shfl_down_sync(0xffffffffu, roots, o);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd((unsigned long long *)&c->parentless, roots);
}

// Every term starts at e = 1 - t without a parent, the batch ends at
// e = 1 - nterms, and there is one parentless symbol per term.
__global__ void k_check(const int32_t *e, const int32_t *par, const long long *offs, long long nterms,
                        const long long *bsum, int nb, Ctl *c)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nterms; t += (long long)gridDim.x * blockDim.x) {
        const long long s = offs[t] - offs[0];
        if (e[s] != 1 - t || par[s] != -1) fail(c);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (1 + bsum[nb] != 1 - nterms) fail(c);
        if (c->parentless != nterms) fail(c);
    }
}

// Records of the batch at slots base .. base + n: head, parent word (sign bit
// for a unary parent), count 1 (tree edge or the root's pin), pending 0,
// argument words beyond the arity and padding 0; each symbol also writes its
// own index into its parent's argument word.  Every record word is written by
// exactly one thread.
__global__ void k_records(DevPool P, const int32_t *flat, const int32_t *e, const int32_t *par, long long n,
                          long long base, int32_t stamp)
{
    const int ma = P.ma, rs = P.rs;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int32_t sym = flat[i];
        const int a = arity_of(P.tab, sym);
        int32_t *r = P.rec + (base + i) * rs;
        const int32_t p = par[i];
        int32_t pw = 0;
        if (p >= 0) {
            const int ap = arity_of(P.tab, flat[p]);
            const int k = ap - 1 - (e[i] - e[p]);
            P.rec[(base + p) * rs + rec_arg(k)] = (int32_t)(base + i);
            pw = (int32_t)((uint32_t)(base + p) | (ap == 1 ? 0x80000000u : 0u));
        }
        r[kRecHead] = sym;
        for (int j = a; j < ma; j++) r[rec_arg(j)] = 0;
        r[rec_par(ma)] = pw;
        r[rec_rc(ma)] = 1;
        r[rec_pend(ma)] = 0;
        for (int w = rec_pend(ma) + 1; w < rs; w++) r[w] = 0;
        P.nfs[base + i] = stamp;
    }
}

}  // namespace up

// ---------------------------------------------------------------------------
// host side

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

cudaError_t scan(long long *v, long long *bsum, dl::Ctl *c, int mode, long long n_fixed, cudaStream_t s)
{
    dl::k_scan_sums<<<dl::kScanBlocks, dl::kThreads, 0, s>>>(v, c, bsum, mode, n_fixed);
    dl::k_scan_top<<<1, 1024, 0, s>>>(bsum, dl::kScanBlocks, c, mode);
    dl::k_scan_apply<<<dl::kScanBlocks, dl::kThreads, 0, s>>>(v, bsum, c, mode, n_fixed);
    return cudaGetLastError();
}

}  // namespace

// Device serialisation of roots[0 .. nroots) (host array) of a pool whose
// high-water mark is n_top, using `scratch` (bytes of device memory that hold
// nothing between normalisations).  Fills offsets_out (nroots + 1) and, if the
// total fits cap, buf.  Returns TRS_OK, TRS_ERR_BUFFER_SMALL, TRS_ERR_STATE
// (dead root or corrupt store), TRS_ERR_TOO_BIG (a subtree deeper than the
// device stacks: the caller serialises on the host instead) or TRS_ERR_CUDA
// with *cuda_err set.
int device_download(const DevPool &P, long long n_top, const int32_t *roots, int nroots, int32_t *buf,
                    int64_t cap, int64_t *offsets_out, void *scratch, size_t scratch_bytes, int num_sms,
                    long long limit_ns, cudaStream_t s, cudaError_t *cuda_err)
{
    constexpr int kRounds = 24;  // unfolding rounds (at most 2^20 items)
    *cuda_err = cudaSuccess;
    char *base = (char *)scratch;
    size_t off = 0;
    auto take = [&](size_t bytes) { char *at = base + off; off = up256(off + bytes); return at; };
    // fixed part: control, buffer pointers, scan block sums
    dl::Ctl *c = (dl::Ctl *)take(sizeof(dl::Ctl));
    int32_t **items_ptr = (int32_t **)take(2 * sizeof(int32_t *));
    int32_t **starts_ptr = (int32_t **)take(2 * sizeof(int32_t *));
    long long *bsum = (long long *)take((dl::kScanBlocks + 1) * sizeof(long long));
    const size_t fixed = off;
    if (scratch_bytes < fixed + 64 * 1024) return TRS_ERR_TOO_BIG;
    const size_t avail = scratch_bytes - fixed;
    // roots per pass and items per pass: at most a third of the scratch area,
    // the rest stages the output
    const long long per_root = 4 + 2 * 4 + 8 + 8;  // roots, 2 x starts, root offsets, spare
    long long rb = (long long)(avail / 8 / per_root);
    if (rb < 1) rb = 1;
    if (rb > nroots) rb = nroots;
    long long m = (long long)((avail / 3 - rb * per_root) / 16);  // 2 x items (4 B) + values (8 B)
    if (m > (1LL << 20)) m = 1LL << 20;
    if (m < rb) return TRS_ERR_TOO_BIG;
    int64_t out_total = 0;
    offsets_out[0] = 0;
    int result = TRS_OK;
    int32_t *items_h[2], *starts_h[2];
    for (int r0 = 0; r0 < nroots; r0 += (int)rb) {
        const int nr = (int)((nroots - r0) < rb ? (nroots - r0) : rb);
        off = fixed;
        int32_t *d_roots = (int32_t *)take((size_t)nr * 4);
        starts_h[0] = (int32_t *)take((size_t)(nr + 1) * 4);
        starts_h[1] = (int32_t *)take((size_t)(nr + 1) * 4);
        long long *roff = (long long *)take((size_t)(nr + 1) * 8);
        items_h[0] = (int32_t *)take((size_t)m * 4);
        items_h[1] = (int32_t *)take((size_t)m * 4);
        long long *vals = (long long *)take((size_t)(m + 1) * 8);
        int32_t *ihead = (int32_t *)take((size_t)m * 4);
        if (off >= scratch_bytes) return TRS_ERR_TOO_BIG;
        // the rest: a third for the output window, two thirds for the chunks
        // the counting walk keeps
        const long long rest = (long long)((scratch_bytes - off) / 4);
        const long long stage_cap = rest / 3 / 64 * 64;
        if (stage_cap < 1024) return TRS_ERR_TOO_BIG;
        int32_t *stage = (int32_t *)take((size_t)stage_cap * 4);
        int32_t *chunks = (int32_t *)(base + off);
        const long long chunk_cap = off < scratch_bytes ? (long long)((scratch_bytes - off) / 4) / dl::kCh : 0;
        const int grid = num_sms * 4;
#define CUDA_STEP(call)                                    \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) { *cuda_err = e_; return TRS_ERR_CUDA; } \
    } while (0)
        CUDA_STEP(cudaMemcpyAsync(items_ptr, items_h, sizeof(items_h), cudaMemcpyHostToDevice, s));
        CUDA_STEP(cudaMemcpyAsync(starts_ptr, starts_h, sizeof(starts_h), cudaMemcpyHostToDevice, s));
        CUDA_STEP(cudaMemsetAsync(c, 0, sizeof(dl::Ctl), s));
        CUDA_STEP(cudaMemcpyAsync(d_roots, roots + r0, (size_t)nr * 4, cudaMemcpyHostToDevice, s));
        dl::k_roots<<<grid, dl::kThreads, 0, s>>>(P, n_top, d_roots, nr, items_h[0], starts_h[0], c);
        CUDA_STEP(cudaGetLastError());
        // unfold the tops of the trees (rounds end as soon as the items
        // would not fit or nothing is left to unfold)
        for (int round = 0; round < kRounds; round++) {
            dl::k_expand_count<<<grid, dl::kThreads, 0, s>>>(P, n_top, items_ptr, vals, c);
            CUDA_STEP(cudaGetLastError());
            CUDA_STEP(scan(vals, bsum, c, 1, 0, s));
            dl::k_expand_write<<<grid, dl::kThreads, 0, s>>>(P, items_ptr, starts_ptr, vals, m, nr, c);
            dl::k_expand_flip<<<1, 1, 0, s>>>(c, m);
            CUDA_STEP(cudaGetLastError());
        }
        // subtree sizes, output offsets, per-root offsets
        dl::k_sizes<<<grid, dl::kThreads, 0, s>>>(P, n_top, items_ptr, vals, c, limit_ns, chunks, chunk_cap, ihead);
        CUDA_STEP(cudaGetLastError());
        CUDA_STEP(scan(vals, bsum, c, 2, 0, s));
        dl::k_root_offsets<<<grid, dl::kThreads, 0, s>>>(starts_ptr, vals, nr, roff, c);
        CUDA_STEP(cudaGetLastError());
        std::vector<long long> ro((size_t)nr + 1);
        dl::Ctl hc;
        CUDA_STEP(cudaMemcpyAsync(ro.data(), roff, ((size_t)nr + 1) * 8, cudaMemcpyDeviceToHost, s));
        CUDA_STEP(cudaMemcpyAsync(&hc, c, sizeof(hc), cudaMemcpyDeviceToHost, s));
        CUDA_STEP(cudaStreamSynchronize(s));
        if (hc.status) return hc.status;
        const long long tot = ro[nr];
        for (int j = 0; j < nr; j++) offsets_out[r0 + j + 1] = out_total + ro[j + 1];
        if (result == TRS_OK && out_total + tot <= cap) {
            for (long long lo = 0; lo < tot; lo += stage_cap) {
                const long long hi = lo + stage_cap < tot ? lo + stage_cap : tot;
                if (hc.overflow)
                    dl::k_emit<<<grid, dl::kThreads, 0, s>>>(P, n_top, items_ptr, vals, stage, lo, hi, c);
                else
                    dl::k_copy<<<grid, dl::kThreads, 0, s>>>(items_ptr, vals, ihead, chunks, stage, lo, hi, c);
                CUDA_STEP(cudaGetLastError());
                CUDA_STEP(cudaMemcpyAsync(buf + out_total + lo, stage, (size_t)(hi - lo) * 4,
                                          cudaMemcpyDeviceToHost, s));
            }
            CUDA_STEP(cudaMemcpyAsync(&hc, c, sizeof(hc), cudaMemcpyDeviceToHost, s));
            CUDA_STEP(cudaStreamSynchronize(s));
            if (hc.status) return hc.status;
        } else {
            result = TRS_ERR_BUFFER_SMALL;  // keep counting: offsets_out gets the sizes
        }
        out_total += tot;
#undef CUDA_STEP
    }
    return result;
}


// Device build of a validated-on-device batch: flat (host, total symbols) and
// offsets (host, nterms + 1) become node records at slots base .. base+total
// of P.  scratch3: three device arrays of at least total int32 each (symbols,
// open places, parents); aux: device bytes for the control word, offsets,
// sparse table and scan sums (aux_bytes, at least upload_aux_bytes()).
// Returns TRS_OK, TRS_ERR_BAD_TERM (nothing written) or TRS_ERR_CUDA.
size_t upload_aux_bytes(long long total, long long nterms)
{
    const long long nch = (total + up::kChunk - 1) / up::kChunk;
    int levels = 1;
    while ((1LL << levels) <= nch) levels++;
    return up256(sizeof(up::Ctl)) + up256((size_t)(nterms + 1) * 8) + up256((size_t)levels * nch * 4) +
           up256((size_t)(up::kScanBlocks + 1) * 8);
}

int device_upload(const DevPool &P, const int32_t *flat, const int64_t *offsets, long long nterms, long long base,
                  int32_t stamp, int32_t *d_flat, int32_t *d_e, int32_t *d_par, void *aux, int num_sms,
                  cudaStream_t s, cudaError_t *cuda_err)
{
    *cuda_err = cudaSuccess;
    const long long total = offsets[nterms] - offsets[0];
    const long long nch = (total + up::kChunk - 1) / up::kChunk;
    int levels = 1;
    while ((1LL << levels) <= nch) levels++;
    char *b = (char *)aux;
    size_t off = 0;
    auto take = [&](size_t bytes) { char *at = b + off; off = up256(off + bytes); return at; };
    up::Ctl *c = (up::Ctl *)take(sizeof(up::Ctl));
    long long *d_offs = (long long *)take((size_t)(nterms + 1) * 8);
    int32_t *st = (int32_t *)take((size_t)levels * nch * 4);
    long long *bsum = (long long *)take((size_t)(up::kScanBlocks + 1) * 8);
    const int grid = num_sms * 4;
    // one thread per symbol for the passes whose threads wait on dependent
    // loads of their own (the resolution of parents outside the chunk, the
    // record writes): with a few threads per symbol range a warp waits for
    // its slowest lane on every round, with one per symbol it retires early
    const long long full = (total + up::kThreads - 1) / up::kThreads;
    const int grid_full = (int)(full < 0x7fffffffLL ? (full > grid ? full : grid) : 0x7fffffffLL);
#define UP_STEP(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) { *cuda_err = e_; return TRS_ERR_CUDA; } \
    } while (0)
    UP_STEP(cudaMemsetAsync(c, 0, sizeof(up::Ctl), s));
    UP_STEP(cudaMemcpyAsync(d_flat, flat + offsets[0], (size_t)total * 4, cudaMemcpyHostToDevice, s));
    UP_STEP(cudaMemcpyAsync(d_offs, offsets, (size_t)(nterms + 1) * 8, cudaMemcpyHostToDevice, s));
    up::k_sums<<<up::kScanBlocks, up::kThreads, 0, s>>>(d_flat, total, P.tab, P.nsym, bsum, c);
    up::k_top<<<1, 1024, 0, s>>>(bsum, up::kScanBlocks);
    up::k_open<<<up::kScanBlocks, up::kThreads, 0, s>>>(d_flat, total, nterms, P.tab, P.nsym, bsum, d_e, c);
    const long long lblocks = (nch + 127) / 128;   // one thread per chunk
    up::k_local<<<(int)(lblocks > grid ? lblocks : grid), 128, 0, s>>>(d_e, total, d_par, st);
    UP_STEP(cudaGetLastError());
    for (int k = 1; k < levels; k++) up::k_table<<<grid, up::kThreads, 0, s>>>(st, nch, k);
    up::k_resolve<<<grid_full, up::kThreads, 0, s>>>(d_e, total, d_par, st, nch, levels, c);
    up::k_check<<<grid, up::kThreads, 0, s>>>(d_e, d_par, d_offs, nterms, bsum, up::kScanBlocks, c);
    UP_STEP(cudaGetLastError());
    up::Ctl hc;
    UP_STEP(cudaMemcpyAsync(&hc, c, sizeof(hc), cudaMemcpyDeviceToHost, s));
    UP_STEP(cudaStreamSynchronize(s));
    if (hc.status != 0) return TRS_ERR_BAD_TERM;
    up::k_records<<<grid_full, up::kThreads, 0, s>>>(P, d_flat, d_e, d_par, total, base, stamp);
    UP_STEP(cudaGetLastError());
#undef UP_STEP
    return TRS_OK;
}

}  // namespace trs
