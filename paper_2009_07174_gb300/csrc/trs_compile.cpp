// trs_compile.cpp -- validation of a TRS and compilation into the rule tables
// the sweep kernels stage into shared memory.  Host only.
//
// Validation follows Def. 1 (a left-hand side is not a variable; the variables
// of a right-hand side occur in its left-hand side) and the left-linearity
// assumption of Sec. 2 (each variable occurs at most once in a left-hand side).
// Compilation replaces the paper's generated rewrite_f functions (Sec. 3, one
// CUDA function per head symbol produced from templates) by data: per rule a
// match program over the left-hand side, a construction program for the
// right-hand side and the net reference-count change of every matched node.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "trs_engine.h"

namespace trs {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

namespace {

struct PNode {            // one node of a parsed preorder term
    int32_t sym;          // > 0 symbol, < 0 variable
    int32_t parent;       // preorder index of the parent, -1 for the root
    int32_t argpos;       // position under the parent
};

// Parse a preorder sequence into nodes; returns TRS_OK or an error.
int parse_preorder(const int32_t *p, int32_t len, int32_t nsym, const std::vector<int32_t> &arity,
                   std::vector<PNode> *out)
{
    out->clear();
    if (!p || len <= 0) return TRS_ERR_ARITY;
    struct Open { int32_t node, next, arity; };
    std::vector<Open> st;
    for (int32_t i = 0; i < len; i++) {
        int32_t s = p[i];
        if (s == 0 || s >= nsym) return TRS_ERR_SYMBOL;
        int32_t parent = -1, argpos = 0;
        if (!st.empty()) {
            parent = st.back().node;
            argpos = st.back().next++;
            if (st.back().next == st.back().arity) st.pop_back();
        } else if (i > 0) {
            return TRS_ERR_ARITY;  // material after a complete term
        }
        out->push_back({s, parent, argpos});
        if (s > 0 && arity[s] > 0) st.push_back({i, 0, arity[s]});
    }
    if (!st.empty()) return TRS_ERR_ARITY;
    return TRS_OK;
}

}  // namespace

int compile_program(const trs_signature *sig, const trs_rule *rules, int32_t nrules,
                    Program *out, std::string *err)
{
    if (!sig || !sig->arity || !out || nrules < 0 || (nrules > 0 && !rules)) {
        *err = "trs_compile: null argument";
        return TRS_ERR_ARG;
    }
    if (sig->nsym < 2 || sig->nsym > TRS_MAX_SYMBOLS) {
        *err = "trs_compile: nsym must be in [2, TRS_MAX_SYMBOLS]";
        return TRS_ERR_MAXARITY;
    }
    if (nrules > TRS_MAX_RULES) {
        *err = "trs_compile: more than TRS_MAX_RULES rules";
        return TRS_ERR_TOO_BIG;
    }
    const int32_t nsym = sig->nsym;
    std::vector<int32_t> arity(sig->arity, sig->arity + nsym);
    arity[0] = 0;
    int32_t ma = 0;
    for (int32_t s = 1; s < nsym; s++) {
        if (arity[s] < 0 || arity[s] > TRS_MAX_ARITY) {
            *err = "trs_compile: arity of symbol " + std::to_string(s) + " out of range";
            return TRS_ERR_MAXARITY;
        }
        ma = std::max(ma, arity[s]);
    }

    struct CRule {
        int32_t orig, head;
        std::vector<uint32_t> pat;
        std::vector<int32_t> build;
        std::vector<int32_t> delta;
        int32_t npat, nnew, rootvar, rootval, root_nargs, root_pend;
    };
    std::vector<CRule> compiled;
    std::vector<PNode> L, R;
    for (int32_t r = 0; r < nrules; r++) {
        const std::string where = "rule " + std::to_string(r) + ": ";
        const trs_rule &ru = rules[r];
        if (!ru.lhs || !ru.rhs || ru.lhs_len <= 0 || ru.rhs_len <= 0) {
            *err = where + "empty side";
            return TRS_ERR_ARG;
        }
        if (ru.lhs[0] < 0) {
            *err = where + "left-hand side is a variable";
            return TRS_ERR_LHS_VAR;
        }
        int st = parse_preorder(ru.lhs, ru.lhs_len, nsym, arity, &L);
        if (st != TRS_OK) { *err = where + "malformed left-hand side"; return st; }
        st = parse_preorder(ru.rhs, ru.rhs_len, nsym, arity, &R);
        if (st != TRS_OK) { *err = where + "malformed right-hand side"; return st; }
        if ((int)L.size() > TRS_MAX_PATTERN || (int)R.size() > TRS_MAX_RHS) {
            *err = where + "side larger than TRS_MAX_PATTERN / TRS_MAX_RHS";
            return TRS_ERR_TOO_BIG;
        }
        // variables of l: each once (left-linear), bound to its pattern register
        std::vector<int32_t> var_reg(TRS_MAX_VARS + 1, -1);
        for (int32_t q = 0; q < (int32_t)L.size(); q++) {
            int32_t s = L[q].sym;
            if (s >= 0) continue;
            int32_t v = -s;
            if (v > TRS_MAX_VARS) { *err = where + "too many variables"; return TRS_ERR_TOO_BIG; }
            if (var_reg[v] >= 0) { *err = where + "variable occurs twice in the left-hand side"; return TRS_ERR_NONLINEAR; }
            var_reg[v] = q;
        }
        for (const PNode &n : R) {
            if (n.sym < 0 && (-n.sym > TRS_MAX_VARS || var_reg[-n.sym] < 0)) {
                *err = where + "right-hand side variable not in the left-hand side";
                return TRS_ERR_RHS_VARS;
            }
        }
        CRule c;
        c.orig = r;
        c.head = L[0].sym;
        c.npat = (int32_t)L.size();
        for (int32_t q = 1; q < c.npat; q++) {
            uint32_t sym = L[q].sym > 0 ? (uint32_t)L[q].sym : 0u;
            c.pat.push_back((uint32_t)L[q].parent | ((uint32_t)L[q].argpos << 8) | (sym << 16));
        }
        // right-hand side: new nodes are the non-root, non-variable positions
        std::vector<int32_t> new_of(R.size(), -1);
        int32_t nnew = 0;
        for (size_t q = 1; q < R.size(); q++)
            if (R[q].sym > 0) new_of[q] = nnew++;
        c.nnew = nnew;
        std::vector<int32_t> occurrences(c.npat, 0);
        auto operand = [&](size_t q) -> int32_t {
            if (R[q].sym < 0) {
                int32_t reg = var_reg[-R[q].sym];
                occurrences[reg]++;
                return reg;
            }
            return new_of[q] | (1 << 16);
        };
        // children of every RHS node, in argument order
        std::vector<std::vector<size_t>> kids(R.size());
        for (size_t q = 1; q < R.size(); q++) kids[R[q].parent].push_back(q);
        if (R[0].sym < 0) {
            c.rootvar = 1;
            c.rootval = var_reg[-R[0].sym];
            c.root_nargs = 0;
            c.root_pend = 0;
        } else {
            c.rootvar = 0;
            c.rootval = R[0].sym;
            c.root_nargs = (int32_t)kids[0].size();
            c.root_pend = 0;
            for (size_t k : kids[0]) {
                c.build.push_back(operand(k));
                if (R[k].sym > 0) c.root_pend++;
            }
        }
        for (size_t q = 1; q < R.size(); q++) {
            if (R[q].sym < 0) continue;
            int32_t pend = 0;
            for (size_t k : kids[q]) if (R[k].sym > 0) pend++;
            int32_t parent_new = R[q].parent == 0 ? -1 : new_of[R[q].parent];
            c.build.push_back(R[q].sym | ((int32_t)kids[q].size() << 16));
            c.build.push_back((parent_new + 1) | (pend << 16));
            for (size_t k : kids[q]) c.build.push_back(operand(k));
        }
        // net reference change per matched node: +1 per new reference from the
        // right-hand side, -1 for each argument of the redex (the redex slot is
        // overwritten, dropping its references; Sec. 3, rewrite listing)
        std::vector<int32_t> net(c.npat, 0);
        for (int32_t q = 1; q < c.npat; q++) {
            net[q] = occurrences[q];
            if (L[q].parent == 0) net[q] -= 1;
        }
        for (int32_t q = 1; q < c.npat; q++)
            if (net[q] > 0) c.delta.push_back(q | (net[q] << 8));
        for (int32_t q = 1; q < c.npat; q++)
            if (net[q] < 0) c.delta.push_back((int32_t)((uint32_t)q | ((uint32_t)net[q] << 8)));
        compiled.push_back(std::move(c));
    }
    // order rule slots by head symbol, keeping textual order inside a head
    std::stable_sort(compiled.begin(), compiled.end(),
                     [](const CRule &a, const CRule &b) { return a.head < b.head; });

    Program p;
    p.nsym = nsym;
    p.maxarity = ma;
    p.nrules = nrules;
    p.arity = arity;
    p.has_rules.assign(nsym, 0);
    std::vector<int32_t> &t = p.table;
    t.assign(8, 0);
    t[0] = kTabMagic; t[1] = nsym; t[2] = ma; t[3] = nrules;
    t[4] = (int32_t)t.size();
    // arity word: arity | prefetch plan << 8.  The plan of a head lists what
    // its patterns read two levels down, so that the matcher can issue those
    // loads together with the argument heads: bit a (a < 4) argument 0 of
    // argument a, bit 4 + a its argument 1, bits 8 + a and 12 + a the head
    // symbols of those two nodes, bit 16 + a the head symbol of argument a.
    std::vector<int32_t> plan(nsym, 0);
    for (const CRule &c : compiled) {
        std::vector<int32_t> par(c.npat, 0), pos(c.npat, 0), depth(c.npat, 0);
        for (int32_t q = 1; q < c.npat; q++) {
            const uint32_t w = (uint32_t)c.pat[q - 1];
            par[q] = (int32_t)(w & 0xff);
            pos[q] = (int32_t)((w >> 8) & 0xff);
            depth[q] = depth[par[q]] + 1;
            if (depth[q] == 1 && pos[q] < 4 && (w >> 16) != 0) plan[c.head] |= 1 << (16 + pos[q]);
            if (depth[q] != 2) continue;
            const int32_t a = pos[par[q]], ap = pos[q];
            const bool sym = (w >> 16) != 0;
            if (a >= 4 || ap >= 2) continue;
            plan[c.head] |= 1 << (4 * ap + a);
            if (sym) plan[c.head] |= 1 << (8 + 4 * ap + a);
        }
    }
    for (int32_t s = 0; s < nsym; s++) t.push_back(arity[s] | (plan[s] << 8));
    t[5] = (int32_t)t.size();
    std::vector<int32_t> first(nsym + 1, 0);
    for (const CRule &c : compiled) first[c.head + 1]++;
    for (int32_t s = 0; s < nsym; s++) first[s + 1] += first[s];
    t.insert(t.end(), first.begin(), first.end());
    t[6] = (int32_t)t.size();
    size_t rules_at = t.size();
    t.resize(t.size() + (size_t)kRuleWords * compiled.size(), 0);
    for (size_t k = 0; k < compiled.size(); k++) {
        const CRule &c = compiled[k];
        p.rule_orig.push_back(c.orig);
        p.has_rules[c.head] = 1;
        int32_t *w = &t[rules_at + (size_t)kRuleWords * k];
        w[0] = c.npat | (c.nnew << 8) | ((int32_t)c.delta.size() << 16) | (c.rootvar << 24);
        w[1] = c.rootval;
        w[2] = (int32_t)t.size();
        for (uint32_t s : c.pat) t.push_back((int32_t)s);
        w = &t[rules_at + (size_t)kRuleWords * k];
        w[3] = (int32_t)t.size();
        t.insert(t.end(), c.build.begin(), c.build.end());
        w = &t[rules_at + (size_t)kRuleWords * k];
        w[4] = (int32_t)t.size();
        t.insert(t.end(), c.delta.begin(), c.delta.end());
        w = &t[rules_at + (size_t)kRuleWords * k];
        w[5] = c.root_nargs | (c.root_pend << 8) | (c.orig << 16);
    }
    t[7] = (int32_t)t.size();
    if ((int)t.size() > kMaxTabWords) {
        *err = "trs_compile: rule tables exceed the shared-memory budget";
        return TRS_ERR_TOO_BIG;
    }
    *out = std::move(p);
    return TRS_OK;
}

}  // namespace trs

extern "C" {

const char *trs_last_error(void) { return trs::g_err.c_str(); }

int trs_compile(const trs_signature *sig, const trs_rule *rules, int32_t nrules,
                trs_program **out)
{
    if (!out) { trs::set_error("trs_compile: out is NULL"); return TRS_ERR_ARG; }
    *out = nullptr;
    trs::Program p;
    std::string err;
    int st = trs::compile_program(sig, rules, nrules, &p, &err);
    if (st != TRS_OK) { trs::set_error(err); return st; }
    trs_program *prog = new trs_program;
    prog->p = std::move(p);
    *out = prog;
    trs::set_error("");
    return TRS_OK;
}

void trs_program_free(trs_program *prog)
{
    if (!prog) return;
    trs::spec_free(prog->spec);
    delete prog;
}

int32_t trs_program_maxarity(const trs_program *prog) { return prog ? prog->p.maxarity : -1; }

}  // extern "C"
