// trs_engine.h -- internal definitions shared by the engine's translation units
// (host compiler, device kernels, C ABI).  Not part of the public ABI.
#pragma once

#include <stdint.h>
#ifndef __CUDACC_RTC__
#include <string>
#include <vector>
#endif

#include "../../include/trs.h"

#ifdef __CUDACC__
#define TRS_HD __host__ __device__
#else
#define TRS_HD
#endif

namespace trs {

// ---------------------------------------------------------------------------
// Compiled rule tables (one int32 word stream, staged into shared memory by
// every kernel that matches rules).
//
//   word 0..7   header: magic, nsym, maxarity, nrules, off_arity, off_first,
//               off_rules, total words
//   arity[nsym]          arity | prefetch plan << 8 (see trs_compile.cpp)
//   first[nsym+1]        rules of head s are rule slots first[s] .. first[s+1]
//   rules[nrules][RW]    per rule slot (in head-symbol order, textual order kept)
//   streams              pattern steps, build program, refcount deltas
//
// Rule slot words:
//   0: npat | nnew << 8 | ndelta << 16 | rootvar << 24
//   1: root symbol (rootvar == 0) or the match register bound to the root
//      variable (rootvar == 1)
//   2: offset of the pattern steps (npat - 1 words)
//   3: offset of the build program
//   4: offset of the refcount deltas (ndelta words)
//   5: root_nargs | root_pend << 8 | original rule index << 16
//
// Pattern step for pattern node q (preorder, q >= 1; register q holds the node
// matched by q, register 0 is the redex itself):
//   parent register | argpos << 8 | symbol << 16   (symbol 0 = a variable)
// Build program: root operands (root_nargs words), then per new node j (RHS
// preorder): [sym | nargs << 16], [parent + 1 | pend << 16], nargs operands.
// parent is -1 for the redex slot, else the index of the parent new node;
// pend counts the new-node arguments (they are not in normal form).
// Operand: index | kind << 16, kind 0 = match register, 1 = new node.
// Delta: register | delta << 8 (arithmetic shift), positive deltas first
// (new references are counted before consumed ones are dropped).
// ---------------------------------------------------------------------------
constexpr int32_t kTabMagic = 0x54525331;  // "TRS1"
constexpr int kRuleWords = 6;
constexpr int kMaxTabWords = 12288;  // 48 KB of shared memory at most

#ifndef __CUDACC_RTC__
struct Program {
    int32_t nsym = 0;
    int32_t maxarity = 0;
    int32_t nrules = 0;
    std::vector<int32_t> arity;
    std::vector<int32_t> table;
    std::vector<int32_t> rule_orig;  // slot -> original rule index
    std::vector<uint8_t> has_rules;  // per symbol
};
#endif

// ---------------------------------------------------------------------------
// Device control block.
// ---------------------------------------------------------------------------
struct Acc {  // per-sweep accumulators, triple-buffered by sweep number % 3
    unsigned long long rewrites, nf_marks, visits, allocs;
    unsigned long long fl_claims;  // allocation positions claimed in this sweep
    unsigned long long deaths;     // reference decrements (each a possible death)
    unsigned long long pushes;     // entries written to the next frontier
    unsigned long long gc_frees, gc_deaths, gc_append;  // garbage collection: freed, dead ones
                                                        // left for the next one, ring appends
    unsigned long long gc_cand;    // garbage collection: candidates taken from the bitmap
    unsigned long long conf_found, refresh_sel;
    unsigned long long taken;      // eager frontier sweep: entries claimed
    unsigned long long pending;    // learned refresh: live nodes not in normal form
    unsigned long long ret;        // allocation positions given back (appended to the ring)
};

struct Ctl {
    // loop state, valid between launches (written by block 0 at exit)
    long long sweep_id;   // number of the next sweep (stamps are relative to it)
    long long n_top;      // high-water mark: slots [1, n_top) have been used
    long long fl_begin;   // free ring: positions [fl_begin, fl_end) hold free slots
    long long fl_end;
    long long dead;       // reference decrements since the last collection (an upper
                          // bound of the dead nodes not yet reclaimed)
    long long fq_size;    // entries in the current frontier
    int fq_cur;           // which frontier buffer is current
    int status;           // trs_status of the device run
    int done;             // graph / host drivers: loop finished
    int gc_pending;       // graph / host drivers: collect before the next sweep
    int mode_phase;       // 1 = seed the frontier at the next launch
    int solo_flags;       // outcome of the last solo episode: done | gc << 1 | confirm << 2 | stop << 3
    int pad0, pad2;
    long long solo_ran;   // sweeps run by the last solo episode
    // statistics of the current trs_normalize
    long long st_rewrites, st_nf_marks, st_sweeps, st_visits, st_allocs, st_frees;
    long long st_gc_runs, st_confirm, st_confirm_found, st_refreshes, st_frontier_peak;
    long long st_solo_sweeps;
    long long sweeps_left;  // max_sweeps budget of the current call
    // grid barrier
    unsigned int bar_count, bar_gen;
    unsigned int solo_gen, pad1;
    long long trace_n;
    long long t_start;      // globaltimer at the start of the current call
    long long since;        // learned: sweeps since the last refresh
    long long samp_n;       // predictor traces: rows written
    Acc acc[3];
};

// Node records.  Slot x occupies rec[x * rs, (x + 1) * rs): its head symbol,
// its ma argument indices, its parent word (frontier modes: the parent of a
// node not in normal form, sign bit set when that parent is unary), its
// reference count and its number of arguments not yet in normal form, then
// padding.  A record is one 32-byte sector up to arity 4 (64 bytes above),
// so one node costs one sector however many of its fields a step touches.
// The normal-form stamps stay a separate array for the streaming scans.
TRS_HD inline int rec_stride(int ma) { return ma + 4 <= 8 ? 8 : 16; }
constexpr int kRecHead = 0;
TRS_HD inline int rec_arg(int a) { return 1 + a; }
TRS_HD inline int rec_par(int ma) { return 1 + ma; }
TRS_HD inline int rec_rc(int ma) { return 2 + ma; }
TRS_HD inline int rec_pend(int ma) { return 3 + ma; }

struct DevPool {
    int32_t *rec;   // node records, rs words per slot
    int32_t *nfs;   // >0: in normal form from sweep nfs; <0: not, eligible from
                    // sweep -nfs; 0: free slot
    int32_t *ring;  // free ring, cap entries, position p at ring[p % cap]
    int32_t *fq[2]; // frontier buffers
    int32_t *act;   // predictor traces: first sweep a node acted after a sample
    uint32_t *dbm;  // candidate bitmap (cap bits): set for a slot whose count was
                    // decremented since the last collection (fire and forget)
    int32_t *cand;  // collection: the candidates compacted from the bitmap
    trs_sweep_record *trace;
    Ctl *ctl;
    const int32_t *tab;  // compiled rule table
    long long cap;
    int32_t ma;
    int32_t rs;     // record stride in words (rec_stride(ma))
    int32_t tab_words;
    int32_t trace_cap;
    int32_t nsym;
    const unsigned char *mlp;  // learned mode: BF16 inference block of the predictor
    int32_t mlp_bytes;
    int32_t pad;
    int32_t *samp_feat;        // predictor traces: rows [h, a_0 .. a_{ma-1}, bits]
    int32_t *samp_slot;
    float *samp_label;
    long long samp_cap;
};

#ifdef __CUDACC__
// ---------------------------------------------------------------------------
// node record accessors (layout above).  The specialised engine compiles
// with the stride and arity as constants.
__device__ __forceinline__ int rec_rs(const DevPool &P)
{
#ifdef TRS_JIT_RS
    return TRS_JIT_RS;
#else
    return P.rs;
#endif
}
__device__ __forceinline__ int rec_ma(const DevPool &P)
{
#ifdef TRS_JIT_MA
    return TRS_JIT_MA;
#else
    return P.ma;
#endif
}
__device__ __forceinline__ int32_t *node_at(const DevPool &P, long long x) { return P.rec + x * rec_rs(P); }
__device__ __forceinline__ int32_t &hs_at(const DevPool &P, long long x) { return node_at(P, x)[kRecHead]; }
__device__ __forceinline__ int32_t &arg_at(const DevPool &P, int a, long long x) { return node_at(P, x)[rec_arg(a)]; }
__device__ __forceinline__ int32_t &par_at(const DevPool &P, long long x) { return node_at(P, x)[rec_par(rec_ma(P))]; }
__device__ __forceinline__ int32_t &rc_at(const DevPool &P, long long x) { return node_at(P, x)[rec_rc(rec_ma(P))]; }
__device__ __forceinline__ int32_t &pend_at(const DevPool &P, long long x) { return node_at(P, x)[rec_pend(rec_ma(P))]; }
// the first four words of a record (head, arguments, ...) in one load
__device__ __forceinline__ int4 rec_head4(const DevPool &P, long long x)
{
    return *reinterpret_cast<const int4 *>(node_at(P, x));
}
// word w (< 4) of a loaded head quadruple
__device__ __forceinline__ int32_t quad_word(const int4 &q, int w)
{
    return w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
}
#endif

constexpr int kTraceCap = 65536;

struct LaunchOpts {
    int32_t mode;
    int32_t block;
    int32_t grid;
    int32_t gc_min_dead;
    int32_t gc_div;
    int32_t solo_max;
    int32_t trace;
    int32_t refresh;
    float threshold;
    int32_t eager;
    long long timeout_ns;
    long long time_limit_ns;
    int32_t sample_period;     // predictor traces: sweeps between samples (0 = off)
    uint32_t sample_thresh;    // sample a node when its hash is below this
    uint32_t sample_seed;
    int32_t pad2;
};

#ifndef __CUDACC_RTC__
// compile (host)
int compile_program(const trs_signature *sig, const trs_rule *rules, int32_t nrules,
                    Program *out, std::string *err);

void set_error(const std::string &msg);

struct SpecEngine;  // the engine compiled for one program (trs_spec.cpp)
void spec_free(SpecEngine *e);
// kernel of the specialised engine for a mode (nullptr: none for this mode)
const void *spec_kernel(const SpecEngine *e, int mode);
#endif

}  // namespace trs

#ifndef __CUDACC_RTC__
struct trs_program {
    trs::Program p;
    trs::SpecEngine *spec = nullptr;
};
#endif
