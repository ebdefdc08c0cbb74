// trs_spec.cpp -- the engine specialised to one rule system.
//
// The paper generates the rewrite code of every head symbol from the rule
// system (Sec. 3: one rewrite function per symbol, emitted from templates).
// trs_specialise does the same at run time: it writes the matcher and the
// rewriter of every rule as straight-line CUDA C++ (spec_decide /
// spec_apply), compiles them together with the engine's own headers with
// NVRTC for the device in use, and loads the result.  The sweep loop, the
// allocation, the collection and the drivers are the table-driven engine's,
// unchanged; only the two functions that interpret the rule tables are
// replaced, so that match registers and new-node slots are addressed by
// constants (registers instead of per-thread memory) and the loads a head's
// patterns need are issued level by level, before any test.
//
// Generated matching, per head symbol h with arguments c_0 .. c_{ar-1}:
//   level 1: the head symbols of the arguments the patterns test and the
//            argument words one level further down, all loaded at once
//            (speculative loads are mapped into the store, see in_store);
//   level 2: the head symbol of a second-level node is loaded just before
//            the first rule that tests it, so that rules decided by level 1
//            alone never wait for it;
//   deeper pattern nodes are loaded inside their rule, in preorder.
// Rules are tested in textual order and the first match wins (Sec. 2).
//
// NVRTC is loaded with dlopen, so that the library itself has no link-time
// dependency on it; the engine's headers are compiled into the library
// (trs_jit_sources.cpp, written by the build), so no source file is read at
// run time.  Compiled images are cached by content hash in an optional
// directory.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "trs_engine.h"

extern "C" {
extern const int trs_jit_source_count;
extern const char *const trs_jit_source_names[];
extern const char *const trs_jit_source_texts[];
}

namespace trs {

namespace {

// ---------------------------------------------------------------------------
// code generation

struct PatNode {
    int parent, argpos, sym;  // sym 0: a variable
    std::vector<int> path;    // argument positions from the redex
};

struct RuleView {
    int slot, npat, nnew, ndelta, rootvar, rootval, root_nargs, root_pend, orig;
    const int32_t *pat, *build, *delta;
};

std::string path_name(const std::vector<int> &p)
{
    std::string s;
    for (size_t t = 0; t < p.size(); t++) s += (t ? "_" : "") + std::to_string(p[t]);
    return s;
}

// value of a pattern node: an argument of the redex, or a deeper node
std::string val_name(const std::vector<int> &p) { return p.size() == 1 ? "c" + path_name(p) : "v" + path_name(p); }
std::string sym_name(const std::vector<int> &p) { return "s" + path_name(p); }

RuleView rule_view(const Program &P, int slot)
{
    const int32_t *t = P.table.data();
    const int32_t *R = t + t[6] + slot * kRuleWords;
    RuleView v;
    v.slot = slot;
    v.npat = R[0] & 0xff;
    v.nnew = (R[0] >> 8) & 0xff;
    v.ndelta = (R[0] >> 16) & 0xff;
    v.rootvar = (R[0] >> 24) & 0xff;
    v.rootval = R[1];
    v.pat = t + R[2];
    v.build = t + R[3];
    v.delta = t + R[4];
    v.root_nargs = R[5] & 0xff;
    v.root_pend = (R[5] >> 8) & 0xff;
    v.orig = (R[5] >> 16) & 0xffff;
    return v;
}

std::vector<PatNode> pattern_nodes(const RuleView &r)
{
    std::vector<PatNode> q(r.npat);
    q[0] = PatNode{-1, -1, 0, {}};
    for (int k = 1; k < r.npat; k++) {
        const uint32_t w = (uint32_t)r.pat[k - 1];
        PatNode n;
        n.parent = (int)(w & 0xff);
        n.argpos = (int)((w >> 8) & 0xff);
        n.sym = (int)(w >> 16);
        n.path = q[n.parent].path;
        n.path.push_back(n.argpos);
        q[k] = n;
    }
    return q;
}

int arity_of(const Program &P, int s) { return (s > 0 && s < P.nsym) ? P.arity[s] : 0; }

// Slot reuse: a constructor argument of the redex that the right-hand side
// does not mention (net reference change -1) dies in the rewrite when the
// redex held its only reference.  Its slot then takes one of the rule's new
// nodes: no allocation, no decrement of it, and its arguments' references
// move to the new nodes (each argument's net change drops by one), so nothing
// is left for the collector.  Whether every paired argument has a count of 1
// is read in the match (the count of a node referenced once cannot change
// during the sweep: only a rewrite of its one parent could touch it), and the
// rule then reuses all pairs or none.
struct ReusePlan {
    std::vector<int> cand;           // pattern registers whose slots are reused, paired with new nodes 0, 1, ...
    std::vector<std::pair<int, int>> delta;  // (register, change) with reuse, positive first
};

ReusePlan reuse_plan(const RuleView &r)
{
    ReusePlan rp;
    const std::vector<PatNode> ns = pattern_nodes(r);
    std::map<int, int> dv;
    for (int d = 0; d < r.ndelta; d++) dv[r.delta[d] & 0xff] = r.delta[d] >> 8;
    for (int q = 1; q < r.npat && (int)rp.cand.size() < r.nnew; q++)
        if (ns[q].parent == 0 && ns[q].sym != 0 && dv.count(q) && dv[q] == -1) rp.cand.push_back(q);
    if (rp.cand.empty()) return rp;
    std::map<int, int> adj = dv;
    for (int c : rp.cand) adj.erase(c);
    for (int q = 1; q < r.npat; q++)
        for (int c : rp.cand)
            if (ns[q].parent == c) adj[q] -= 1;
    for (auto &e : adj)
        if (e.second > 0) rp.delta.push_back(e);
    for (auto &e : adj)
        if (e.second < 0) rp.delta.push_back(e);
    return rp;
}


// Arguments whose records the decision for head h loads (their heads or
// second-level words appear in h's patterns, or their counts decide a slot
// reuse).  When a rewrite makes a node of head h its continuation, the
// records of these arguments are prefetched, so that the next step's
// dependent load hits L1.
std::set<int> inspected_args(const Program &P, int h)
{
    std::set<int> out;
    if (h <= 0 || h >= P.nsym) return out;
    const int32_t *first = P.table.data() + P.table[5];
    for (int s = first[h]; s < first[h + 1]; s++) {
        const RuleView r = rule_view(P, s);
        const std::vector<PatNode> ns = pattern_nodes(r);
        for (size_t q = 1; q < ns.size(); q++) {
            if (ns[q].path.size() == 1 && ns[q].sym) out.insert(ns[q].path[0]);
            if (ns[q].path.size() == 2 && ns[q].path[1] < 3) out.insert(ns[q].path[0]);
        }
        for (int q : reuse_plan(r).cand) out.insert(ns[q].argpos);
    }
    return out;
}

void gen_decide_head(std::ostringstream &o, const Program &P, int h, int first, int last)
{
    const int ar = arity_of(P, h);
    o << "    case " << h << ": {\n";
    for (int j = 0; j < ar; j++) {
        if (j < 4) o << "        const int32_t c" << j << " = w" << j << ";\n";
        else o << "        const int32_t c" << j << " = arg_at(P, " << j << ", i);\n";
    }
    if (ar > 0) {
        o << "        if (check_ready) {\n            bool ready = true;\n";
        for (int j = 0; j < ar; j++) o << "            ready &= nf_ready(P, c" << j << ", k, check_ready);\n";
        o << "            if (!ready) return D_SKIP;\n        }\n";
    }
    // every pattern node of every rule of h, by path
    std::vector<RuleView> rules;
    std::vector<std::vector<PatNode>> nodes;
    for (int s = first; s < last; s++) {
        rules.push_back(rule_view(P, s));
        nodes.push_back(pattern_nodes(rules.back()));
    }
    std::set<std::vector<int>> sym1, val2;
    for (auto &ns : nodes)
        for (size_t q = 1; q < ns.size(); q++) {
            const PatNode &n = ns[q];
            if (n.path.size() == 1 && n.sym) sym1.insert(n.path);
            if (n.path.size() == 2) val2.insert(n.path);
        }
    // argument positions whose counts decide a slot reuse
    std::set<int> rcpos;
    std::vector<ReusePlan> plans;
    for (size_t ri = 0; ri < rules.size(); ri++) {
        plans.push_back(reuse_plan(rules[ri]));
        for (int q : plans.back().cand) rcpos.insert(nodes[ri][q].argpos);
    }
    // level 1: argument heads and second-level words together, one load of
    // the first four record words per argument (the count is in the same
    // sector)
    std::set<int> quad;
    for (auto &p : sym1) quad.insert(p[0]);
    for (auto &p : val2)
        if (p[1] < 3) quad.insert(p[0]);
    for (int j : quad) o << "        const int4 n" << j << " = rec_head4(P, c" << j << ");\n";
    for (int j : rcpos) o << "        const int32_t rc" << j << " = rc_at(P, c" << j << ");\n";
    for (auto &p : sym1) o << "        const int32_t " << sym_name(p) << " = n" << p[0] << ".x;\n";
    for (auto &p : val2) {
        if (p[1] < 3)
            o << "        const int32_t " << val_name(p) << " = in_store(n" << p[0] << "." << "yzw"[p[1]] << ", cap);\n";
        else
            o << "        const int32_t " << val_name(p) << " = in_store(arg_at(P, " << p[1] << ", c" << p[0] << "), cap);\n";
    }
    std::set<std::vector<int>> emitted;
    for (size_t ri = 0; ri < rules.size(); ri++) {
        const RuleView &r = rules[ri];
        const std::vector<PatNode> &ns = nodes[ri];
        // level 2: head symbols this rule tests, loaded just before its test
        for (size_t q = 1; q < ns.size(); q++)
            if (ns[q].path.size() == 2 && ns[q].sym && !emitted.count(ns[q].path)) {
                emitted.insert(ns[q].path);
                o << "        const int32_t " << sym_name(ns[q].path) << " = hs_at(P, " << val_name(ns[q].path) << ");\n";
            }
        o << "        do {  // rule " << r.orig << "\n";
        std::string cond;
        for (size_t q = 1; q < ns.size(); q++)
            if (ns[q].path.size() <= 2 && ns[q].sym) {
                if (!cond.empty()) cond += " || ";
                cond += sym_name(ns[q].path) + " != " + std::to_string(ns[q].sym);
            }
        if (!cond.empty()) o << "            if (" << cond << ") break;\n";
        for (size_t q = 1; q < ns.size(); q++) {
            const PatNode &n = ns[q];
            if (n.path.size() <= 2) continue;
            std::vector<int> pp(n.path.begin(), n.path.end() - 1);
            o << "            const int32_t " << val_name(n.path) << " = arg_at(P, " << n.argpos << ", "
              << val_name(pp) << ");\n";
            if (n.sym) o << "            if (hs_at(P, " << val_name(n.path) << ") != " << n.sym << ") break;\n";
        }
        o << "            reg[0] = i;\n";
        for (size_t q = 1; q < ns.size(); q++) o << "            reg[" << q << "] = " << val_name(ns[q].path) << ";\n";
        // decision word: rule slot | reuse << 16 | slots to allocate << 17
        if (plans[ri].cand.empty()) {
            o << "            return " << (r.slot | (r.nnew << 17)) << ";\n        } while (0);\n";
        } else {
            std::string u;
            for (int q : plans[ri].cand) u += std::string(u.empty() ? "" : " && ") + "rc" + std::to_string(ns[q].argpos) + " == 1";
            const int with = r.slot | 0x10000 | ((r.nnew - (int)plans[ri].cand.size()) << 17);
            const int without = r.slot | (r.nnew << 17);
            o << "            return (" << u << ") ? " << with << " : " << without << ";\n        } while (0);\n";
        }
    }
    o << "        return D_MARK;\n    }\n";
}

void gen_apply_body(std::ostringstream &o, const Program &P, const RuleView &r, const ReusePlan *rp)
{
    int pos = r.root_nargs;
    std::vector<int> new_sym;
    // the slot of new node j as an expression
    auto new_slot = [&](int j) -> std::string {
        const int np = rp ? (int)rp->cand.size() : 0;
        return j < np ? "reg[" + std::to_string(rp->cand[j]) + "]" : "nw[" + std::to_string(j - np) + "]";
    };
    // an operand: a match register or the slot of a new node
    auto opnd = [&](int32_t op) -> std::string {
        return (op >> 16) ? new_slot(op & 0xffff) : "reg[" + std::to_string(op & 0xffff) + "]";
    };
    // the content of a node that becomes the eager continuation (its
    // arguments' records are prefetched for the next step)
    auto emit_carry = [&](const std::string &ind, int sym, const std::vector<std::string> &ops,
                          const std::string &parw) {
        const int na = (int)ops.size();
        for (int a : inspected_args(P, sym))
            if (a < na) o << ind << "prefetch_rec(P, " << ops[a] << ");\n";
        if (na <= 4) {
            o << ind << "last.h = " << sym << ";\n";
            for (int a = 0; a < na; a++) o << ind << "last.c[" << a << "] = " << ops[a] << ";\n";
            o << ind << "last.p = " << parw << ";\n";
        } else {
            o << ind << "last.h = 0;\n";
        }
    };
    // learned mode queues the nodes a rewrite makes ready, the eager
    // continuation last; a redex that waits for new arguments is queued by
    // the last of them to become a normal form
    for (int j = 0; j < r.nnew; j++) {
        const int32_t w0 = r.build[pos++], w1 = r.build[pos++];
        const int sym = w0 & 0xffff, na = w0 >> 16;
        const int parent = (w1 & 0xffff) - 1, pj = w1 >> 16;
        new_sym.push_back(sym);
        const int npairs = rp ? (int)rp->cand.size() : 0;
        if (j < npairs)
            o << "        {\n            const int32_t x = reg[" << rp->cand[j] << "];\n";
        else
            o << "        {\n            const int32_t x = nw[" << j - npairs << "];\n";
        std::vector<std::string> ops;
        for (int a = 0; a < na; a++) ops.push_back(opnd(r.build[pos++]));
        std::string parw;
        if (parent < 0) {
            const bool un = arity_of(P, r.rootval) == 1;
            parw = std::string("i") + (un ? " | (int32_t)0x80000000" : "");
        } else {
            const bool un = arity_of(P, new_sym[parent]) == 1;
            parw = new_slot(parent) + (un ? " | (int32_t)0x80000000" : "");
        }
        // the whole record in 16-byte stores: head, arguments, parent word,
        // count 1, pending arguments (learned mode: the sweep it was queued for)
        const int ma = P.maxarity, rs = rec_stride(ma);
        std::vector<std::string> w(rs, "0");
        w[kRecHead] = std::to_string(sym);
        for (int a = 0; a < na; a++) w[rec_arg(a)] = ops[a];
        w[rec_par(ma)] = "(" + parw + ")";
        w[rec_rc(ma)] = "1";
        // learned mode: a node queued for the next sweep carries that sweep's
        // number; one waiting for new arguments is queued by the last of them
        w[rec_pend(ma)] = pj == 0 ? "(mode == M_LEARNED ? (int32_t)(k + 1) : 0)"
                                  : "(mode == M_LEARNED ? 0 : " + std::to_string(pj) + ")";
        for (int q = 0; q < rs; q += 4)
            o << "            reinterpret_cast<int4 *>(node_at(P, x))[" << q / 4 << "] = make_int4(" << w[q] << ", "
              << w[q + 1] << ", " << w[q + 2] << ", " << w[q + 3] << ");\n";
        o << "            P.nfs[x] = stamp_new;\n";
        o << "            if (mode == M_LEARNED) {\n";
        if (pj == 0) {
            o << "                push[npush++] = x;\n";
            emit_carry("                ", sym, ops, "(" + parw + ")");
        }
        o << "            } else {\n";
        if (pj == 0) {
            o << "                if (mode == M_FRONTIER) {\n                    push[npush++] = x;\n";
            emit_carry("                    ", sym, ops, "(" + parw + ")");
            o << "                }\n";
        }
        o << "            }\n        }\n";
    }
    const int ma = P.maxarity;
    if (r.rootvar) {
        o << "        const int32_t x = reg[" << r.rootval << "];\n        const int4 xq = rec_head4(P, x);\n"
             "        const int32_t xh = xq.x;\n";
        for (int a = 0; a < ma; a++) {
            if (a < 3) o << "        const int32_t xc" << a << " = xq." << "yzw"[a] << ";\n";
            else o << "        const int32_t xc" << a << " = arg_at(P, " << a << ", x);\n";
        }
        o << "        const int xa = T.arity(xh);\n";
        for (int a = 0; a < ma; a++) o << "        if (" << a << " < xa) red_add_s32(&rc_at(P, xc" << a << "), 1);\n";
    }
    std::vector<std::pair<int, int>> deltas;
    if (rp) {
        deltas = rp->delta;
    } else {
        for (int d = 0; d < r.ndelta; d++) deltas.push_back({r.delta[d] & 0xff, r.delta[d] >> 8});
    }
    // fire and forget: a decremented node becomes a collection candidate
    for (auto &e : deltas) {
        o << "        red_add_s32(&rc_at(P, reg[" << e.first << "]), " << e.second << ");\n";
        if (e.second < 0) o << "        mark_candidate(P, reg[" << e.first << "], C);\n";
    }
    if (r.rootvar) {
        o << "        hs_at(P, i) = xh;\n";
        for (int a = 0; a < ma; a++) o << "        if (" << a << " < xa) arg_at(P, " << a << ", i) = xc" << a << ";\n";
        o << "        store_nf(P, mode, i, k);\n        {\n            const int before = npush;\n"
             "            if (mode == M_FRONTIER) notify_parent(P, pv, push, npush);\n"
             "            if (mode == M_LEARNED) {\n                const int32_t p = pv & 0x7fffffff;\n"
             "                if (p != 0) learned_push(P, p, k + 1, push, npush);\n            }\n"
             "            if (npush != before) last.h = 0;\n        }\n";
    } else {
        o << "        hs_at(P, i) = " << r.rootval << ";\n";
        std::vector<std::string> ops;
        for (int a = 0; a < r.root_nargs; a++) {
            ops.push_back(opnd(r.build[a]));
            o << "        arg_at(P, " << a << ", i) = " << ops.back() << ";\n";
        }
        o << "        if (mode == M_LEARNED) {\n"
             "            st_release_s32(&P.nfs[i], -(int32_t)(k + 1));\n";
        if (r.root_pend == 0) {
            // the redex is this lane's: queued (or continued) without a claim
            o << "            pend_at(P, i) = (int32_t)(k + 1);\n            push[npush++] = i;\n";
            emit_carry("            ", r.rootval, ops, "pv");
        }
        o << "        } else {\n            pend_at(P, i) = " << r.root_pend << ";\n";
        if (r.root_pend == 0) {
            o << "            if (mode == M_FRONTIER) {\n                push[npush++] = i;\n";
            emit_carry("                ", r.rootval, ops, "pv");
            o << "            }\n";
        }
        o << "        }\n";
    }
    if (r.nnew) o << "        C.allocs += " << r.nnew << ";\n";
}

void gen_apply_rule(std::ostringstream &o, const Program &P, const RuleView &r)
{
    o << "    case " << r.slot << ": {  // rule " << r.orig << "\n";
    const ReusePlan rp = reuse_plan(r);
    if (rp.cand.empty()) {
        gen_apply_body(o, P, r, nullptr);
    } else {
        o << "      if (reuse) {\n";
        gen_apply_body(o, P, r, &rp);
        o << "      } else {\n";
        gen_apply_body(o, P, r, nullptr);
        o << "      }\n";
    }
    o << "        break;\n    }\n";
}

std::string generate(const Program &P)
{
    std::ostringstream o;
    const int32_t *t = P.table.data();
    const int32_t *first = t + t[5];
    const int mw = P.maxarity < 4 ? P.maxarity : 4;
    o << "// generated from the rule tables: " << P.nrules << " rules over " << P.nsym - 1 << " symbols\n";
    o << "namespace trs {\n\n";
    o << "__device__ __forceinline__ int spec_decide(const DevPool &P, const Tab &T, int32_t i, long long k,\n"
         "                                           int check_ready, int32_t *reg, int32_t &h_out,\n"
         "                                           const Carry &cin)\n{\n";
    o << "    const long long cap = P.cap;\n    int32_t h;\n";
    for (int j = 0; j < 4; j++) o << "    int32_t w" << j << " = 0;\n";
    o << "    if (cin.h != 0) {\n        h = cin.h;\n";
    for (int j = 0; j < mw; j++) o << "        w" << j << " = cin.c[" << j << "];\n";
    o << "    } else {\n        const int4 q = rec_head4(P, i);\n        h = q.x;\n";
    for (int j = 0; j < mw; j++) {
        if (j < 3) o << "        w" << j << " = q." << "yzw"[j] << ";\n";
        else o << "        w" << j << " = arg_at(P, " << j << ", i);\n";
    }
    o << "    }\n    h_out = h;\n    switch (h) {\n";
    for (int h = 1; h < P.nsym; h++)
        if (first[h + 1] > first[h]) gen_decide_head(o, P, h, first[h], first[h + 1]);
    o << "    default:\n        break;\n    }\n";
    // heads without rules: a normal form once the arguments are
    o << "    if (check_ready) {\n        const int ar = T.arity(h);\n        bool ready = true;\n";
    for (int j = 0; j < P.maxarity; j++) {
        const std::string w = j < 4 ? "w" + std::to_string(j) : "arg_at(P, " + std::to_string(j) + ", i)";
        o << "        if (" << j << " < ar) ready &= nf_ready(P, " << w << ", k, check_ready);\n";
    }
    o << "        if (!ready) return D_SKIP;\n    }\n    return D_MARK;\n}\n\n";

    o << "__device__ __forceinline__ void spec_apply(const DevPool &P, const Tab &T, int mode, int32_t i, int32_t h,\n"
         "                                           int32_t pv, int r, long long k, const int32_t *reg,\n"
         "                                           const int32_t *nw, Counters &C, int32_t *push, int &npush,\n"
         "                                           Carry &last)\n{\n";
    o << "    last.h = 0;\n    if (r == D_MARK) {\n        apply_mark(P, mode, i, pv, k, C, push, npush);\n        return;\n    }\n";
    o << "    const long long cap = P.cap;\n    const int32_t stamp_new = -(int32_t)(k + 1);\n    (void)stamp_new;\n";
    o << "    const bool reuse = (r >> 16) & 1;\n    (void)reuse;\n";
    o << "    switch (r & 0xffff) {\n";
    for (int s = 0; s < (int)P.rule_orig.size(); s++) gen_apply_rule(o, P, rule_view(P, s));
    o << "    default:\n        break;\n    }\n";
    o << "    if (P.act) P.act[i] = min(P.act[i], (int32_t)k);\n    C.rewrites++;\n}\n\n";
    // slots to allocate for a decision (new nodes not placed in reused slots)
    o << "__device__ __forceinline__ int spec_new_count(int d)\n{\n    return (d >> 17) & 0xff;\n}\n\n"
         "}  // namespace trs\n";
    return o.str();
}

// ---------------------------------------------------------------------------
// NVRTC, loaded at run time

struct Nvrtc {
    void *lib = nullptr;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcAddNameExpression) add_name = nullptr;
    decltype(&nvrtcGetLoweredName) lowered = nullptr;
    decltype(&nvrtcVersion) version = nullptr;
};

bool load_nvrtc(Nvrtc &n, std::string *err)
{
    static std::mutex mu;
    static Nvrtc cached;
    static bool tried = false;
    std::lock_guard<std::mutex> lock(mu);
    if (!tried) {
        tried = true;
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        for (const char *nm : names) {
            cached.lib = dlopen(nm, RTLD_NOW | RTLD_LOCAL);
            if (cached.lib) break;
        }
        if (cached.lib) {
#define TRS_SYM(field, name) cached.field = (decltype(cached.field))dlsym(cached.lib, name)
            TRS_SYM(create, "nvrtcCreateProgram");
            TRS_SYM(compile, "nvrtcCompileProgram");
            TRS_SYM(log_size, "nvrtcGetProgramLogSize");
            TRS_SYM(log, "nvrtcGetProgramLog");
            TRS_SYM(cubin_size, "nvrtcGetCUBINSize");
            TRS_SYM(cubin, "nvrtcGetCUBIN");
            TRS_SYM(destroy, "nvrtcDestroyProgram");
            TRS_SYM(add_name, "nvrtcAddNameExpression");
            TRS_SYM(lowered, "nvrtcGetLoweredName");
            TRS_SYM(version, "nvrtcVersion");
#undef TRS_SYM
        }
    }
    if (!cached.lib || !cached.create || !cached.compile || !cached.cubin || !cached.lowered) {
        *err = "trs_specialise: NVRTC (libnvrtc.so) not found";
        return false;
    }
    n = cached;
    return true;
}

// FNV-1a, 64 bit: cache key of a compiled image
uint64_t fnv(const std::string &s, uint64_t h = 1469598103934665603ull)
{
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

std::string cuda_include_dir()
{
    const char *env[] = {"TRS_CUDA_INCLUDE", nullptr};
    for (int t = 0; env[t]; t++) {
        const char *v = getenv(env[t]);
        if (v && *v) return v;
    }
    const char *home = getenv("CUDA_HOME");
    if (home && *home) return std::string(home) + "/include";
    return "/usr/local/cuda/include";
}

const char *kStdint =
    "#pragma once\n"
    "typedef signed char int8_t; typedef short int16_t; typedef int int32_t; typedef long long int64_t;\n"
    "typedef unsigned char uint8_t; typedef unsigned short uint16_t; typedef unsigned int uint32_t;\n"
    "typedef unsigned long long uint64_t; typedef unsigned long long uintptr_t; typedef long long intptr_t;\n";
const char *kStddef = "#pragma once\ntypedef unsigned long size_t; typedef long ptrdiff_t;\n";

const char *kModeNames[3] = {"trs::k_engine<0>", "trs::k_engine<1>", "trs::k_engine<2>"};

}  // namespace

struct SpecEngine {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern[3] = {nullptr, nullptr, nullptr};
    std::string source;  // the generated rule code
    std::string log;     // compiler log (resources per kernel)
};

void spec_free(SpecEngine *e)
{
    if (!e) return;
    if (e->lib) cudaLibraryUnload(e->lib);
    delete e;
}

const void *spec_kernel(const SpecEngine *e, int mode)
{
    if (!e || mode < 0 || mode > 2) return nullptr;
    return (const void *)e->kern[mode];
}

}  // namespace trs

using namespace trs;

extern "C" {

}  // extern "C"

namespace {

// Generate and compile the engine for `prog` and architecture sm_<cc>a, or
// take it from the cache; fills image, the lowered kernel names and the log.
int compile_spec(const trs_program *prog, int cc, const char *cache_dir, std::vector<char> &image,
                 std::string lowered[3], std::string &gen, std::string &log)
{
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(cc) + "a";
    gen = generate(prog->p);
    const std::string src = "#define TRS_JIT 1\n#define TRS_JIT_MA " + std::to_string(prog->p.maxarity) +
                            "\n#define TRS_JIT_RS " + std::to_string(rec_stride(prog->p.maxarity)) +
                            "\n#include \"trs_device.cuh\"\n" + gen + "#include \"trs_engine_kernel.cuh\"\n";
    const std::string inc = "-I" + cuda_include_dir();
    std::vector<std::string> opts = {arch, "-std=c++17", "-default-device", inc, "--ptxas-options=-v"};
    // cache key: generated code, engine sources, options
    uint64_t key = fnv(src);
    for (int t = 0; t < trs_jit_source_count; t++)
        key = fnv(trs_jit_source_texts[t], fnv(trs_jit_source_names[t], key));
    for (const std::string &s : opts) key = fnv(s, key);
    char keyhex[32];
    snprintf(keyhex, sizeof keyhex, "%016llx", (unsigned long long)key);
    std::string cache_path;
    if (cache_dir && *cache_dir) cache_path = std::string(cache_dir) + "/spec_" + keyhex + ".bin";
    image.clear();
    if (!cache_path.empty()) {
        std::ifstream in(cache_path, std::ios::binary);
        if (in) {
            // cache file: three lowered names (one per line), then the image
            for (int m = 0; m < 3; m++) std::getline(in, lowered[m]);
            image.assign(std::istreambuf_iterator<char>(in), std::istreambuf_iterator<char>());
            if (image.empty() || lowered[0].empty() || lowered[1].empty() || lowered[2].empty()) image.clear();
            if (!image.empty()) return TRS_OK;
        }
    }
    Nvrtc nv;
    std::string err;
    if (!load_nvrtc(nv, &err)) { set_error(err); return TRS_ERR_JIT; }
    std::vector<const char *> hdr, names;
    for (int t = 0; t < trs_jit_source_count; t++) {
        hdr.push_back(trs_jit_source_texts[t]);
        names.push_back(trs_jit_source_names[t]);
    }
    hdr.push_back(kStdint);
    names.push_back("stdint.h");
    hdr.push_back(kStddef);
    names.push_back("stddef.h");
    nvrtcProgram np;
    nvrtcResult r = nv.create(&np, src.c_str(), "trs_spec.cu", (int)hdr.size(), hdr.data(), names.data());
    if (r != NVRTC_SUCCESS) { set_error("trs_specialise: nvrtcCreateProgram failed"); return TRS_ERR_JIT; }
    for (int m = 0; m < 3; m++) nv.add_name(np, kModeNames[m]);
    std::vector<const char *> o;
    for (const std::string &s : opts) o.push_back(s.c_str());
    r = nv.compile(np, (int)o.size(), o.data());
    size_t ls = 0;
    nv.log_size(np, &ls);
    if (ls > 1) {
        std::vector<char> buf(ls);
        nv.log(np, buf.data());
        log.assign(buf.data());
    }
    if (r != NVRTC_SUCCESS) {
        nv.destroy(&np);
        set_error("trs_specialise: compile error:\n" + log.substr(0, 6000));
        return TRS_ERR_JIT;
    }
    size_t cs = 0;
    nv.cubin_size(np, &cs);
    image.resize(cs);
    nv.cubin(np, image.data());
    for (int m = 0; m < 3; m++) {
        const char *ln = nullptr;
        nv.lowered(np, kModeNames[m], &ln);
        lowered[m] = ln ? ln : "";
    }
    nv.destroy(&np);
    if (!cache_path.empty()) {
        const std::string tmp = cache_path + ".tmp" + std::to_string((long long)getpid());
        std::ofstream out(tmp, std::ios::binary);
        if (out) {
            for (int m = 0; m < 3; m++) out << lowered[m] << "\n";
            out.write(image.data(), (std::streamsize)image.size());
            out.close();
            std::rename(tmp.c_str(), cache_path.c_str());
        }
    }
    return TRS_OK;
}

}  // namespace

extern "C" {

int trs_specialise(trs_program *prog, const char *cache_dir)
{
    if (!prog) { set_error("trs_specialise: program is NULL"); return TRS_ERR_ARG; }
    if (prog->spec) return TRS_OK;
    int dev = 0, maj = 0, mnr = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
    if (ce != cudaSuccess) {
        set_error(std::string("trs_specialise: no CUDA device: ") + cudaGetErrorString(ce));
        return TRS_ERR_CUDA;
    }
    std::vector<char> image;
    std::string lowered[3], gen, log;
    int st = compile_spec(prog, maj * 10 + mnr, cache_dir, image, lowered, gen, log);
    if (st != TRS_OK) return st;
    SpecEngine *e = new SpecEngine;
    e->source = gen;
    e->log = log;
    ce = cudaLibraryLoadData(&e->lib, image.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    for (int m = 0; m < 3 && ce == cudaSuccess; m++)
        ce = cudaLibraryGetKernel(&e->kern[m], e->lib, lowered[m].c_str());
    if (ce != cudaSuccess) {
        set_error(std::string("trs_specialise: loading the compiled engine failed: ") + cudaGetErrorString(ce));
        spec_free(e);
        return TRS_ERR_CUDA;
    }
    prog->spec = e;
    set_error("");
    return TRS_OK;
}

int trs_specialise_compile(const trs_program *prog, int32_t cc, const char *cache_dir, int64_t *image_bytes)
{
    if (!prog || cc <= 0) { set_error("trs_specialise_compile: bad argument"); return TRS_ERR_ARG; }
    std::vector<char> image;
    std::string lowered[3], gen, log;
    int st = compile_spec(prog, cc, cache_dir, image, lowered, gen, log);
    if (st != TRS_OK) return st;
    if (image_bytes) *image_bytes = (int64_t)image.size();
    set_error(log);
    return TRS_OK;
}

int trs_program_is_specialised(const trs_program *prog) { return prog && prog->spec ? 1 : 0; }

int64_t trs_specialised_source(const trs_program *prog, char *buf, int64_t cap)
{
    if (!prog) return -1;
    const std::string s = prog->spec ? prog->spec->source : generate(prog->p);
    if (buf && cap > 0) {
        const size_t n = std::min((size_t)cap - 1, s.size());
        std::memcpy(buf, s.data(), n);
        buf[n] = 0;
    }
    return (int64_t)s.size() + 1;
}

}  // extern "C"
