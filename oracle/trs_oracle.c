/*
 * trs_oracle.c -- plain CPU term rewriter used as the parity oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA engine.
 *
 * Terms are ordinary pointer trees (one heap node per symbol occurrence, no
 * sharing, no reference counts, no garbage collector): a variable that occurs
 * twice in a right-hand side is deep-copied, a variable that does not occur is
 * freed.  Three strategies are provided:
 *
 *   mode 0  leftmost-innermost derivation: the recursive procedure `derive` /
 *           `rewrite_f` of Sec. 2 (Listing "derivation procedure"), run with an
 *           explicit stack because terms are tens of thousands of levels deep.
 *           Rules of a head symbol are tried in the given order and the first
 *           match is applied (Sec. 2, the rewrite procedure); a term none of
 *           whose rules match is marked as normal form.
 *   mode 1  leftmost-outermost: repeatedly rewrite the first redex in preorder
 *           (used only to check that the normal form does not depend on the
 *           strategy for the confluent workloads; Sec. 2 strategy discussion).
 *   mode 2  synchronous parallel innermost: in each sweep every term that is not
 *           in normal form and whose subterms all are is rewritten (or marked as
 *           normal form), all against the state at the start of the sweep
 *           (Sec. 3: the derive kernel reads nf_read, a per-iteration copy of
 *           nf).  A new right-hand-side term starts not-in-normal-form; a term
 *           replaced by a variable's (normal-form) binding is in normal form at
 *           once, as in the paper's Plus(Zero,X) -> X example.  Counts sweeps.
 *
 * Statistics returned: rewrites (successful rule applications, the paper's
 * "rewritten terms"), nf marks (terms concluded to be in normal form because no
 * rule matched), sweeps (mode 2: sweeps in which something happened; modes 0/1:
 * 0) and the peak number of live nodes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXAR 8
#define OR_MAXVARS 64

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_STEPS = 2, OR_ERR_BUF = 3, OR_ERR_OOM = 4 };

typedef struct onode {
    int32_t sym;
    int32_t nf;
    struct onode *ch[]; /* arity(sym) children */
} onode;

typedef struct {
    int32_t *lhs; int32_t lhs_len;
    int32_t *rhs; int32_t rhs_len;
    int32_t nvars;
} orule;

typedef struct otrs {
    int32_t nsym;
    int32_t *arity;
    int32_t nrules;
    orule *rules;
    int32_t *first;   /* rules of symbol s: by_sym[first[s] .. first[s+1]) */
    int32_t *by_sym;
    /* node allocator: one free list per arity */
    onode *freelist[OR_MAXAR + 1];
    void **chunks; int64_t nchunks, capchunks;
    int64_t live, peak;
    int oom;
} otrs;

/* ------------------------------------------------------------------------- */
/* node allocation                                                           */

static onode *node_new(otrs *o, int32_t sym)
{
    int a = o->arity[sym];
    onode *n = o->freelist[a];
    if (n) {
        o->freelist[a] = n->ch[0];
    } else {
        size_t sz = sizeof(onode) + sizeof(onode *) * (size_t)(a > 0 ? a : 1);
        n = (onode *)malloc(sz);
        if (!n) { o->oom = 1; return NULL; }
        if (o->nchunks == o->capchunks) {
            int64_t nc = o->capchunks ? 2 * o->capchunks : 1024;
            void **p = (void **)realloc(o->chunks, sizeof(void *) * (size_t)nc);
            if (!p) { free(n); o->oom = 1; return NULL; }
            o->chunks = p; o->capchunks = nc;
        }
        o->chunks[o->nchunks++] = n;
    }
    n->sym = sym;
    n->nf = 0;
    for (int i = 0; i < a; i++) n->ch[i] = NULL;
    if (++o->live > o->peak) o->peak = o->live;
    return n;
}

static void node_release(otrs *o, onode *n)
{
    int a = o->arity[n->sym];
    /* arity-0 nodes still own one pointer slot for the free-list link */
    n->ch[0] = o->freelist[a];
    o->freelist[a] = n;
    o->live--;
}

/* free a whole tree (iteratively: trees are deep) */
static void tree_free(otrs *o, onode *t)
{
    if (!t) return;
    int64_t cap = 256, sp = 0;
    onode **st = (onode **)malloc(sizeof(onode *) * (size_t)cap);
    st[sp++] = t;
    while (sp) {
        onode *n = st[--sp];
        int a = o->arity[n->sym];
        for (int i = 0; i < a; i++) {
            if (sp == cap) { cap *= 2; st = (onode **)realloc(st, sizeof(onode *) * (size_t)cap); }
            st[sp++] = n->ch[i];
        }
        node_release(o, n);
    }
    free(st);
}

/* deep copy (iteratively) */
static onode *tree_copy(otrs *o, onode *t)
{
    onode *root = NULL;
    int64_t cap = 256, sp = 0;
    onode ***dst = (onode ***)malloc(sizeof(onode **) * (size_t)cap);
    onode **src = (onode **)malloc(sizeof(onode *) * (size_t)cap);
    dst[sp] = &root; src[sp] = t; sp++;
    while (sp) {
        sp--;
        onode *s = src[sp];
        onode **d = dst[sp];
        onode *n = node_new(o, s->sym);
        if (!n) break;
        n->nf = s->nf;
        *d = n;
        int a = o->arity[s->sym];
        for (int i = 0; i < a; i++) {
            if (sp == cap) {
                cap *= 2;
                dst = (onode ***)realloc(dst, sizeof(onode **) * (size_t)cap);
                src = (onode **)realloc(src, sizeof(onode *) * (size_t)cap);
            }
            dst[sp] = &n->ch[i]; src[sp] = s->ch[i]; sp++;
        }
    }
    free(dst); free(src);
    return root;
}

/* ------------------------------------------------------------------------- */
/* term <-> preorder                                                          */

static onode *tree_from_preorder(otrs *o, const int32_t *pre, int64_t len)
{
    if (len <= 0) return NULL;
    onode *root = NULL;
    int64_t cap = 256, sp = 0, pos = 0;
    onode ***slot = (onode ***)malloc(sizeof(onode **) * (size_t)cap);
    slot[sp++] = &root;
    int bad = 0;
    while (sp) {
        onode **d = slot[--sp];
        if (pos >= len) { bad = 1; break; }
        int32_t s = pre[pos++];
        if (s <= 0 || s >= o->nsym) { bad = 1; break; }
        onode *n = node_new(o, s);
        if (!n) { bad = 1; break; }
        *d = n;
        int a = o->arity[s];
        for (int i = a - 1; i >= 0; i--) { /* push right-to-left: leftmost first */
            if (sp == cap) { cap *= 2; slot = (onode ***)realloc(slot, sizeof(onode **) * (size_t)cap); }
            slot[sp++] = &n->ch[i];
        }
    }
    free(slot);
    if (bad || pos != len) { /* partial trees have NULL holes: release carefully */
        /* fill holes so tree_free is safe */
        if (root) {
            int64_t c2 = 256, s2 = 0;
            onode **st = (onode **)malloc(sizeof(onode *) * (size_t)c2);
            st[s2++] = root;
            while (s2) {
                onode *n = st[--s2];
                int a = o->arity[n->sym];
                for (int i = 0; i < a; i++) {
                    if (n->ch[i]) {
                        if (s2 == c2) { c2 *= 2; st = (onode **)realloc(st, sizeof(onode *) * (size_t)c2); }
                        st[s2++] = n->ch[i];
                    }
                }
                /* children already pushed; detach and release this node */
                for (int i = 0; i < a; i++) n->ch[i] = NULL;
                node_release(o, n);
            }
            free(st);
        }
        return NULL;
    }
    return root;
}

static int64_t tree_to_preorder(otrs *o, onode *t, int32_t *out, int64_t cap)
{
    int64_t n = 0, scap = 256, sp = 0;
    onode **st = (onode **)malloc(sizeof(onode *) * (size_t)scap);
    st[sp++] = t;
    while (sp) {
        onode *x = st[--sp];
        if (n < cap) out[n] = x->sym;
        n++;
        int a = o->arity[x->sym];
        for (int i = a - 1; i >= 0; i--) {
            if (sp == scap) { scap *= 2; st = (onode **)realloc(st, sizeof(onode *) * (size_t)scap); }
            st[sp++] = x->ch[i];
        }
    }
    free(st);
    return n;
}

/* ------------------------------------------------------------------------- */
/* matching and instantiation (patterns are small: plain recursion)           */

/* Match pattern pat[*pos..] against t; bind variables (left-linear: each
 * variable occurs once).  Sec. 2: l matches t iff some substitution sigma has
 * l sigma = t. */
static int match(const otrs *o, const int32_t *pat, int32_t *pos, onode *t, onode **bind)
{
    int32_t s = pat[(*pos)++];
    if (s < 0) { bind[-s - 1] = t; return 1; }
    int a = o->arity[s];
    if (t->sym != s) {
        /* skip the rest of this pattern subtree */
        int need = a;
        while (need > 0) { int32_t q = pat[(*pos)++]; need--; if (q > 0) need += o->arity[q]; }
        return 0;
    }
    int ok = 1;
    for (int i = 0; i < a; i++) {
        if (ok) ok = match(o, pat, pos, t->ch[i], bind);
        else {
            int need = 1;
            while (need > 0) { int32_t q = pat[(*pos)++]; need--; if (q > 0) need += o->arity[q]; }
        }
    }
    return ok;
}

/* Build r sigma.  The first use of a variable moves its binding, later uses
 * deep-copy it. */
static onode *instantiate(otrs *o, const int32_t *rhs, int32_t *pos, onode **bind, int32_t *used)
{
    int32_t s = rhs[(*pos)++];
    if (s < 0) {
        int v = -s - 1;
        if (used[v]++ == 0) return bind[v];
        return tree_copy(o, bind[v]);
    }
    onode *n = node_new(o, s);
    if (!n) return NULL;
    int a = o->arity[s];
    for (int i = 0; i < a; i++) n->ch[i] = instantiate(o, rhs, pos, bind, used);
    return n;
}

/* Release the nodes matched by the non-variable positions of the pattern. */
static void free_skeleton(otrs *o, const int32_t *pat, int32_t *pos, onode *t)
{
    int32_t s = pat[(*pos)++];
    if (s < 0) return;
    int a = o->arity[s];
    for (int i = 0; i < a; i++) free_skeleton(o, pat, pos, t->ch[i]);
    node_release(o, t);
}

/* Try the rules of hs(t) in order (first match wins).  Returns the rule index
 * applied, or -1.  On success *loc holds r sigma and the old term is gone. */
static int rewrite_at(otrs *o, onode **loc)
{
    onode *t = *loc;
    onode *bind[OR_MAXVARS];
    int32_t used[OR_MAXVARS];
    for (int k = o->first[t->sym]; k < o->first[t->sym + 1]; k++) {
        int ri = o->by_sym[k];
        const orule *r = &o->rules[ri];
        int32_t pos = 0;
        if (!match(o, r->lhs, &pos, t, bind)) continue;
        for (int v = 0; v < r->nvars; v++) used[v] = 0;
        pos = 0;
        onode *res = instantiate(o, r->rhs, &pos, bind, used);
        pos = 0;
        free_skeleton(o, r->lhs, &pos, t);
        for (int v = 0; v < r->nvars; v++)
            if (used[v] == 0) tree_free(o, bind[v]);
        *loc = res;
        return ri;
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* strategies                                                                 */

typedef struct { int64_t rewrites, nf_marks, sweeps; } ostats;

void otrs_destroy(otrs *o);

/* mode 0: Listing "derivation procedure" with an explicit stack of locations. */
static int run_innermost(otrs *o, onode **root, int64_t cap, ostats *st, int64_t *rc)
{
    int64_t scap = 1024, sp = 0;
    onode ***stk = (onode ***)malloc(sizeof(onode **) * (size_t)scap);
    stk[sp++] = root;
    int status = OR_OK;
    while (sp) {
        onode **loc = stk[sp - 1];
        onode *t = *loc;
        if (t->nf) { sp--; continue; }
        int a = o->arity[t->sym], j;
        for (j = 0; j < a; j++) if (!t->ch[j]->nf) break;
        if (j < a) {                              /* derive a subterm first */
            if (sp == scap) { scap *= 2; stk = (onode ***)realloc(stk, sizeof(onode **) * (size_t)scap); }
            stk[sp++] = &t->ch[j];
            continue;
        }
        int ri = rewrite_at(o, loc);               /* all subterms in normal form */
        if (ri < 0) { t->nf = 1; st->nf_marks++; sp--; continue; }
        if (o->oom) { status = OR_ERR_OOM; break; }
        st->rewrites++;
        if (rc) rc[ri]++;
        if (cap >= 0 && st->rewrites >= cap) { status = OR_ERR_STEPS; break; }
    }
    free(stk);
    return status;
}

/* mode 1: leftmost-outermost.  nf here means "no redex anywhere below". */
static int first_match_rule(const otrs *o, onode *t)
{
    onode *bind[OR_MAXVARS];
    for (int k = o->first[t->sym]; k < o->first[t->sym + 1]; k++) {
        int32_t pos = 0;
        if (match(o, o->rules[o->by_sym[k]].lhs, &pos, t, bind)) return o->by_sym[k];
    }
    return -1;
}

static int run_outermost(otrs *o, onode **root, int64_t cap, ostats *st, int64_t *rc)
{
    int64_t scap = 1024;
    onode ***loc = (onode ***)malloc(sizeof(onode **) * (size_t)scap);
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)scap);
    int status = OR_OK;
    for (;;) {
        int64_t sp = 0;
        onode **redex = NULL;
        loc[sp] = root; nxt[sp] = -1; sp++;
        while (sp) {
            onode *t = *loc[sp - 1];
            if (nxt[sp - 1] == -1) {
                if (t->nf) { sp--; continue; }
                if (first_match_rule(o, t) >= 0) { redex = loc[sp - 1]; break; }
                nxt[sp - 1] = 0;
            }
            int a = o->arity[t->sym];
            if (nxt[sp - 1] < a) {
                int c = nxt[sp - 1]++;
                if (sp == scap) {
                    scap *= 2;
                    loc = (onode ***)realloc(loc, sizeof(onode **) * (size_t)scap);
                    nxt = (int32_t *)realloc(nxt, sizeof(int32_t) * (size_t)scap);
                }
                loc[sp] = &t->ch[c]; nxt[sp] = -1; sp++;
                continue;
            }
            t->nf = 1;
            sp--;
        }
        if (!redex) break;
        int ri = rewrite_at(o, redex);
        if (o->oom) { status = OR_ERR_OOM; break; }
        st->rewrites++;
        if (rc) rc[ri]++;
        if (cap >= 0 && st->rewrites >= cap) { status = OR_ERR_STEPS; break; }
    }
    free(loc); free(nxt);
    return status;
}

/* mode 2: synchronous sweeps.  The ready set of a sweep is collected before any
 * of it is rewritten, so every decision uses the state at the sweep's start. */
static int run_parallel(otrs *o, onode **root, int64_t cap, ostats *st, int64_t *rc)
{
    int64_t scap = 1024, rcap = 1024;
    onode ***stk = (onode ***)malloc(sizeof(onode **) * (size_t)scap);
    onode ***ready = (onode ***)malloc(sizeof(onode **) * (size_t)rcap);
    int status = OR_OK;
    for (;;) {
        int64_t sp = 0, nr = 0;
        stk[sp++] = root;
        while (sp) {
            onode **l = stk[--sp];
            onode *t = *l;
            if (t->nf) continue;
            int a = o->arity[t->sym], all = 1;
            for (int j = 0; j < a; j++) {
                if (!t->ch[j]->nf) {
                    all = 0;
                    if (sp == scap) { scap *= 2; stk = (onode ***)realloc(stk, sizeof(onode **) * (size_t)scap); }
                    stk[sp++] = &t->ch[j];
                }
            }
            if (all) {
                if (nr == rcap) { rcap *= 2; ready = (onode ***)realloc(ready, sizeof(onode **) * (size_t)rcap); }
                ready[nr++] = l;
            }
        }
        if (nr == 0) break;
        st->sweeps++;
        /* nf marks made in this sweep become visible in the next one */
        onode **marked = (onode **)malloc(sizeof(onode *) * (size_t)nr);
        int64_t nm = 0;
        for (int64_t i = 0; i < nr; i++) {
            onode *t = *ready[i];
            int ri = rewrite_at(o, ready[i]);
            if (ri < 0) { marked[nm++] = t; continue; }
            if (o->oom) { status = OR_ERR_OOM; break; }
            st->rewrites++;
            if (rc) rc[ri]++;
        }
        for (int64_t i = 0; i < nm; i++) marked[i]->nf = 1;
        st->nf_marks += nm;
        free(marked);
        if (status != OR_OK) break;
        if (cap >= 0 && st->sweeps >= cap) { status = OR_ERR_STEPS; break; }
    }
    free(stk); free(ready);
    return status;
}

/* ------------------------------------------------------------------------- */
/* public API (ctypes)                                                        */

static int pattern_ok(const int32_t *p, int32_t len, int32_t nsym, const int32_t *arity, int32_t *maxvar)
{
    int32_t need = 1, i;
    for (i = 0; i < len && need > 0; i++) {
        int32_t s = p[i];
        need--;
        if (s < 0) {
            if (-s > OR_MAXVARS) return 0;
            if (-s > *maxvar) *maxvar = -s;
            continue;
        }
        if (s == 0 || s >= nsym) return 0;
        if (arity[s] > OR_MAXAR) return 0;
        need += arity[s];
    }
    return need == 0 && i == len;
}

otrs *otrs_create(int32_t nsym, const int32_t *arity, int32_t nrules,
                  const int32_t *lhs_flat, const int64_t *lhs_off,
                  const int32_t *rhs_flat, const int64_t *rhs_off)
{
    if (nsym < 2 || nrules < 0) return NULL;
    otrs *o = (otrs *)calloc(1, sizeof(otrs));
    o->nsym = nsym;
    o->arity = (int32_t *)malloc(sizeof(int32_t) * (size_t)nsym);
    memcpy(o->arity, arity, sizeof(int32_t) * (size_t)nsym);
    o->nrules = nrules;
    o->rules = (orule *)calloc((size_t)(nrules > 0 ? nrules : 1), sizeof(orule));
    for (int r = 0; r < nrules; r++) {
        orule *q = &o->rules[r];
        q->lhs_len = (int32_t)(lhs_off[r + 1] - lhs_off[r]);
        q->rhs_len = (int32_t)(rhs_off[r + 1] - rhs_off[r]);
        q->lhs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(q->lhs_len + 1));
        q->rhs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(q->rhs_len + 1));
        memcpy(q->lhs, lhs_flat + lhs_off[r], sizeof(int32_t) * (size_t)q->lhs_len);
        memcpy(q->rhs, rhs_flat + rhs_off[r], sizeof(int32_t) * (size_t)q->rhs_len);
        int32_t mv = 0, mv2 = 0;
        if (!pattern_ok(q->lhs, q->lhs_len, nsym, arity, &mv) || q->lhs[0] < 0 ||
            !pattern_ok(q->rhs, q->rhs_len, nsym, arity, &mv2) || mv2 > mv) {
            o->nrules = r + 1;
            otrs_destroy(o);
            return NULL;
        }
        q->nvars = mv;
    }
    o->first = (int32_t *)calloc((size_t)nsym + 1, sizeof(int32_t));
    o->by_sym = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nrules > 0 ? nrules : 1));
    for (int r = 0; r < nrules; r++) o->first[o->rules[r].lhs[0] + 1]++;
    for (int s = 0; s < nsym; s++) o->first[s + 1] += o->first[s];
    int32_t *fill = (int32_t *)calloc((size_t)nsym, sizeof(int32_t));
    for (int r = 0; r < nrules; r++) {          /* stable: textual order kept */
        int s = o->rules[r].lhs[0];
        o->by_sym[o->first[s] + fill[s]++] = r;
    }
    free(fill);
    return o;
}

void otrs_destroy(otrs *o)
{
    if (!o) return;
    for (int r = 0; r < o->nrules; r++) { free(o->rules[r].lhs); free(o->rules[r].rhs); }
    free(o->rules); free(o->arity); free(o->first); free(o->by_sym);
    for (int64_t i = 0; i < o->nchunks; i++) free(o->chunks[i]);
    free(o->chunks);
    free(o);
}

/* stats[0..3] = rewrites, nf marks, sweeps, peak live nodes.  rule_counts
 * (nrules entries) may be NULL.  step_cap < 0 means unlimited (rewrites for
 * modes 0/1, sweeps for mode 2). */
int otrs_normalize(otrs *o, int32_t mode, const int32_t *term, int64_t len, int64_t step_cap,
                   int32_t *out, int64_t out_cap, int64_t *out_len, int64_t *stats,
                   int64_t *rule_counts)
{
    if (!o || !term || len <= 0 || mode < 0 || mode > 2) return OR_ERR_ARG;
    o->oom = 0;
    o->live = 0; o->peak = 0;
    onode *root = tree_from_preorder(o, term, len);
    if (!root) return o->oom ? OR_ERR_OOM : OR_ERR_ARG;
    ostats st = {0, 0, 0};
    if (rule_counts) memset(rule_counts, 0, sizeof(int64_t) * (size_t)o->nrules);
    int status;
    if (mode == 0) status = run_innermost(o, &root, step_cap, &st, rule_counts);
    else if (mode == 1) status = run_outermost(o, &root, step_cap, &st, rule_counts);
    else status = run_parallel(o, &root, step_cap, &st, rule_counts);
    if (stats) { stats[0] = st.rewrites; stats[1] = st.nf_marks; stats[2] = st.sweeps; stats[3] = o->peak; }
    if (status == OR_OK) {
        int64_t n = tree_to_preorder(o, root, out, out_cap);
        if (out_len) *out_len = n;
        if (n > out_cap) status = OR_ERR_BUF;
    }
    tree_free(o, root);
    return status;
}
