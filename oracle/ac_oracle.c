/*
 * Oracle for exact multiple-pattern matching — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library. The product (the CUDA scan behind include/ac.h) never
 * links, calls or includes anything from here, and this file shares no code,
 * header, table or helper with it.
 *
 * What it computes. For patterns P_0..P_{P-1} (byte strings, ids = their index
 * in the input array) and a text t[0..n), the result is the set
 *     M = { (e, j) : |P_j| <= e+1 <= n  and  t[e-|P_j|+1 .. e] = P_j }
 * sorted by end position e (0-based, inclusive), then by pattern id j, plus
 * counts[j] = |{ e : (e, j) in M }|.
 *
 * Three independent routes to M live here:
 *   oracle_scan   — the Aho-Corasick machine with failure links as Section II.A
 *                   of the paper describes it (Fig. 1): a goto function made by
 *                   inserting the patterns one after another, numbering new
 *                   states consecutively from root 0; a failure function; an
 *                   output function. The text is read one character at a time;
 *                   when the current state has no valid transition for the
 *                   character, the machine follows failure transitions and
 *                   considers the same character again, and whenever it is in a
 *                   final state it produces that state's patterns.
 *                   The failure function is computed breadth-first and the
 *                   output of a state is merged with the output of its failure
 *                   state (the classical construction of reference [1]; the
 *                   paper relies on it when state 2 fails to state 4 on 'E').
 *   oracle_pfac   — the failure-less machine of Section II.B / Section IV.A
 *                   (Figs. 2-4, Fig. 6): the same goto function without failure
 *                   transitions; a walk starts at every text position from
 *                   state 0 and stops at the first missing transition,
 *                   producing the pattern of every final state it passes.
 *   oracle_brute  — the definition of M written out: compare every pattern
 *                   against the text ending at every position.
 *
 * Parity is pinned (see tests/test_oracle.py) by the paper's worked examples
 * (Fig. 1 "ABEDE", Fig. 6 "USHERS", with the state numbers the text quotes),
 * by agreement of the three routes on thousands of random small cases, by a
 * closed form (all k-mers), and by compiling deliberately broken variants
 * (ORACLE_MUTANT=k) and checking that each one fails a pin.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define FAIL UINT32_MAX

typedef struct {
    uint8_t sym;
    uint32_t to;
} oedge;

typedef struct {
    oedge *edge;        /* goto transitions leaving this state, in creation order */
    uint32_t nedge, capedge;
    uint32_t fail;      /* failure function f(s) */
    uint32_t *own;      /* patterns whose last character leads here (final state) */
    uint32_t nown, capown;
    uint32_t *out;      /* output function: own patterns plus those of f(s) */
    uint32_t nout;
    uint32_t depth;
} ostate;

typedef struct oracle_machine {
    ostate *st;
    uint32_t ns, cap;
    uint32_t P;
    uint32_t maxlen;
    int with_failure;
} oracle_machine;

typedef struct {
    uint32_t *v;   /* pairs: v[2i] = end position, v[2i+1] = pattern id */
    uint64_t n, cap;
    int oom;
} pairbuf;

static void pb_push(pairbuf *b, uint32_t pos, uint32_t id) {
    if (b->oom) return;
    if (b->n == b->cap) {
        uint64_t nc = b->cap ? 2 * b->cap : 1024;
        uint32_t *nv = (uint32_t *)realloc(b->v, (size_t)nc * 2 * sizeof(uint32_t));
        if (!nv) { b->oom = 1; return; }
        b->v = nv;
        b->cap = nc;
    }
    b->v[2 * b->n] = pos;
    b->v[2 * b->n + 1] = id;
    b->n++;
}

static int cmp_pair(const void *a, const void *b) {
    const uint32_t *x = (const uint32_t *)a, *y = (const uint32_t *)b;
#if ORACLE_MUTANT == 6
    /* planted mistake: order by id first */
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
#else
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
#endif
    return 0;
}

static uint32_t new_state(oracle_machine *m, uint32_t depth) {
    if (m->ns == m->cap) {
        uint32_t nc = m->cap ? 2 * m->cap : 64;
        ostate *n2 = (ostate *)realloc(m->st, (size_t)nc * sizeof(ostate));
        if (!n2) return FAIL;
        m->st = n2;
        m->cap = nc;
    }
    ostate *s = &m->st[m->ns];
    memset(s, 0, sizeof(*s));
    s->fail = 0;
    s->depth = depth;
    return m->ns++;
}

static int add_u32(uint32_t **arr, uint32_t *n, uint32_t *cap, uint32_t x) {
    if (*n == *cap) {
        uint32_t nc = *cap ? 2 * *cap : 2;
        uint32_t *na = (uint32_t *)realloc(*arr, (size_t)nc * sizeof(uint32_t));
        if (!na) return -1;
        *arr = na;
        *cap = nc;
    }
    (*arr)[(*n)++] = x;
    return 0;
}

/* g(s, c) restricted to explicit transitions: FAIL when there is none. */
static uint32_t edge_to(const oracle_machine *m, uint32_t s, uint8_t c) {
    const ostate *q = &m->st[s];
    for (uint32_t i = 0; i < q->nedge; i++)
        if (q->edge[i].sym == c) return q->edge[i].to;
    return FAIL;
}

/* The goto function of the failure-link machine: the root has a transition
 * back to itself on every character that does not start a pattern, so the
 * failure loop always ends there. */
static uint32_t g(const oracle_machine *m, uint32_t s, uint8_t c) {
    uint32_t t = edge_to(m, s, c);
    if (t == FAIL && s == 0) return 0;
    return t;
}

void oracle_free(oracle_machine *m) {
    if (!m) return;
    for (uint32_t i = 0; i < m->ns; i++) {
        free(m->st[i].edge);
        free(m->st[i].own);
        free(m->st[i].out);
    }
    free(m->st);
    free(m);
}

/* Build the machine. with_failure = 0 builds the failure-less machine of
 * Section II.B (goto and final states only). Returns 0, or -1 on bad input
 * (P = 0 or an empty pattern), or -2 when out of memory. */
int oracle_build(const uint8_t *const *pats, const uint32_t *lens, uint32_t P,
                 int with_failure, oracle_machine **out) {
    *out = NULL;
    if (P == 0) return -1;
    for (uint32_t j = 0; j < P; j++)
        if (lens[j] == 0 || !pats[j]) return -1;
    oracle_machine *m = (oracle_machine *)calloc(1, sizeof(*m));
    if (!m) return -2;
    m->P = P;
    m->with_failure = with_failure;
    if (new_state(m, 0) == FAIL) { oracle_free(m); return -2; }

    /* goto function: insert each pattern in the given order */
    for (uint32_t j = 0; j < P; j++) {
        uint32_t s = 0;
        if (lens[j] > m->maxlen) m->maxlen = lens[j];
        for (uint32_t k = 0; k < lens[j]; k++) {
            uint8_t c = pats[j][k];
            uint32_t t = edge_to(m, s, c);
            if (t == FAIL) {
                t = new_state(m, m->st[s].depth + 1);
                if (t == FAIL) { oracle_free(m); return -2; }
                ostate *q = &m->st[s];
                if (q->nedge == q->capedge) {
                    uint32_t nc = q->capedge ? 2 * q->capedge : 2;
                    oedge *ne = (oedge *)realloc(q->edge, nc * sizeof(oedge));
                    if (!ne) { oracle_free(m); return -2; }
                    q->edge = ne;
                    q->capedge = nc;
                }
                q->edge[q->nedge].sym = c;
                q->edge[q->nedge].to = t;
                q->nedge++;
            }
            s = t;
        }
        if (add_u32(&m->st[s].own, &m->st[s].nown, &m->st[s].capown, j)) {
            oracle_free(m);
            return -2;
        }
    }

    /* output function starts as the own patterns of each final state */
    for (uint32_t s = 0; s < m->ns; s++) {
        ostate *q = &m->st[s];
        if (q->nown) {
            q->out = (uint32_t *)malloc(q->nown * sizeof(uint32_t));
            if (!q->out) { oracle_free(m); return -2; }
            memcpy(q->out, q->own, q->nown * sizeof(uint32_t));
            q->nout = q->nown;
        }
    }
    if (!with_failure) { *out = m; return 0; }

    /* failure function, breadth first */
    uint32_t *queue = (uint32_t *)malloc((size_t)m->ns * sizeof(uint32_t));
    if (!queue) { oracle_free(m); return -2; }
    uint32_t head = 0, tail = 0;
    for (uint32_t i = 0; i < m->st[0].nedge; i++) {
        uint32_t t = m->st[0].edge[i].to;
        m->st[t].fail = 0;
        queue[tail++] = t;
    }
    while (head < tail) {
        uint32_t r = queue[head++];
        for (uint32_t i = 0; i < m->st[r].nedge; i++) {
            uint8_t a = m->st[r].edge[i].sym;
            uint32_t t = m->st[r].edge[i].to;
            queue[tail++] = t;
#if ORACLE_MUTANT == 3
            /* planted mistake: every failure goes to the root */
            uint32_t f = 0;
#elif ORACLE_MUTANT == 5
            /* planted mistake: look only one failure level up */
            uint32_t f = g(m, m->st[r].fail, a);
            if (f == FAIL) f = 0;
#else
            uint32_t state = m->st[r].fail;
            while (g(m, state, a) == FAIL) state = m->st[state].fail;
            uint32_t f = g(m, state, a);
#endif
            m->st[t].fail = f;
#if ORACLE_MUTANT != 1
            /* output(t) := output(t) ∪ output(f(t)); f(t) is shallower, so
             * its output is already complete */
            ostate *qt = &m->st[t], *qf = &m->st[f];
            if (qf->nout) {
                uint32_t *no = (uint32_t *)realloc(qt->out, (size_t)(qt->nout + qf->nout) * sizeof(uint32_t));
                if (!no) { free(queue); oracle_free(m); return -2; }
                memcpy(no + qt->nout, qf->out, qf->nout * sizeof(uint32_t));
                qt->out = no;
                qt->nout += qf->nout;
            }
#endif
        }
    }
    free(queue);
    *out = m;
    return 0;
}

uint32_t oracle_num_states(const oracle_machine *m) { return m->ns; }
uint32_t oracle_max_len(const oracle_machine *m) { return m->maxlen; }
uint32_t oracle_fail(const oracle_machine *m, uint32_t s) { return s < m->ns ? m->st[s].fail : FAIL; }
uint32_t oracle_depth(const oracle_machine *m, uint32_t s) { return s < m->ns ? m->st[s].depth : FAIL; }
uint32_t oracle_goto(const oracle_machine *m, uint32_t s, uint8_t c) { return s < m->ns ? edge_to(m, s, c) : FAIL; }

/* state reached after reading a string from the root along goto edges */
uint32_t oracle_state_of(const oracle_machine *m, const uint8_t *str, uint32_t len) {
    uint32_t s = 0;
    for (uint32_t k = 0; k < len && s != FAIL; k++) s = edge_to(m, s, str[k]);
    return s;
}

/* one step of the failure-link machine on character c */
static uint32_t step(const oracle_machine *m, uint32_t s, uint8_t c) {
#if ORACLE_MUTANT == 4
    /* planted mistake: on a failure, drop the character instead of
     * considering it again in the failure state */
    if (g(m, s, c) == FAIL) return m->st[s].fail;
    return g(m, s, c);
#else
    while (g(m, s, c) == FAIL) s = m->st[s].fail;
    return g(m, s, c);
#endif
}

static void emit_state(const oracle_machine *m, uint32_t s, uint64_t i, pairbuf *b) {
    const ostate *q = &m->st[s];
    for (uint32_t k = 0; k < q->nout; k++) {
#if ORACLE_MUTANT == 2
        pb_push(b, (uint32_t)(i + 1), q->out[k]);   /* planted mistake: off by one */
#else
        pb_push(b, (uint32_t)i, q->out[k]);
#endif
    }
}

/* the state after each character (Fig. 1 trace) */
int oracle_trace(const oracle_machine *m, const uint8_t *text, uint64_t n, uint32_t *states) {
    if (!m->with_failure) return -1;
    uint32_t s = 0;
    for (uint64_t i = 0; i < n; i++) {
        s = step(m, s, text[i]);
        states[i] = s;
    }
    return 0;
}

/* Scan text[start..end) from the root and keep matches ending in
 * [emit_lo, end). Used whole (start = emit_lo = 0) by oracle_scan and per
 * chunk by oracle_scan_mt. */
static void scan_range(const oracle_machine *m, const uint8_t *text, uint64_t start,
                       uint64_t emit_lo, uint64_t end, pairbuf *b) {
    uint32_t s = 0;
    for (uint64_t i = start; i < end; i++) {
        s = step(m, s, text[i]);
        if (i >= emit_lo && m->st[s].nout) emit_state(m, s, i, b);
    }
}

static int finish(pairbuf *b, uint32_t **pairs, uint64_t *M) {
    if (b->oom) { free(b->v); *pairs = NULL; *M = 0; return -2; }
    if (b->n) qsort(b->v, (size_t)b->n, 2 * sizeof(uint32_t), cmp_pair);
    *pairs = b->v;
    *M = b->n;
    return 0;
}

int oracle_scan(const oracle_machine *m, const uint8_t *text, uint64_t n,
                uint32_t **pairs, uint64_t *M) {
    if (!m->with_failure) return -1;
    pairbuf b = {0};
    scan_range(m, text, 0, 0, n, &b);
    return finish(&b, pairs, M);
}

/* Input-focused split across POSIX threads (Section III, the first of the two
 * architectures of [2]): chunk c owns end positions [s_c, e_c) and starts
 * from the root at max(0, s_c - (maxlen - 1)). */
typedef struct {
    const oracle_machine *m;
    const uint8_t *text;
    uint64_t start, lo, hi;
    pairbuf b;
} mt_job;

static void *mt_run(void *arg) {
    mt_job *j = (mt_job *)arg;
    scan_range(j->m, j->text, j->start, j->lo, j->hi, &j->b);
    return NULL;
}

int oracle_scan_mt(const oracle_machine *m, const uint8_t *text, uint64_t n, int nthreads,
                   uint32_t **pairs, uint64_t *M) {
    if (!m->with_failure) return -1;
    if (nthreads < 1) nthreads = 1;
    mt_job *jobs = (mt_job *)calloc((size_t)nthreads, sizeof(mt_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    uint64_t chunk = (n + nthreads - 1) / (uint64_t)nthreads;
    uint64_t warm = m->maxlen ? m->maxlen - 1 : 0;
    for (int c = 0; c < nthreads; c++) {
        uint64_t lo = (uint64_t)c * chunk, hi = lo + chunk;
        if (lo > n) lo = n;
        if (hi > n) hi = n;
        jobs[c].m = m;
        jobs[c].text = text;
        jobs[c].lo = lo;
        jobs[c].hi = hi;
        jobs[c].start = lo > warm ? lo - warm : 0;
        pthread_create(&th[c], NULL, mt_run, &jobs[c]);
    }
    pairbuf all = {0};
    for (int c = 0; c < nthreads; c++) {
        pthread_join(th[c], NULL);
        if (jobs[c].b.oom) all.oom = 1;
        for (uint64_t k = 0; k < jobs[c].b.n; k++) pb_push(&all, jobs[c].b.v[2 * k], jobs[c].b.v[2 * k + 1]);
        free(jobs[c].b.v);
    }
    free(jobs);
    free(th);
    return finish(&all, pairs, M);
}

/* Failure-less walk from one start position (Fig. 4 / Fig. 6): the states
 * visited until the first missing transition. Returns how many were visited
 * (at most cap are stored). */
uint64_t oracle_pfac_walk(const oracle_machine *m, const uint8_t *text, uint64_t n,
                          uint64_t start, uint32_t *states, uint64_t cap) {
    uint32_t s = 0;
    uint64_t k = 0;
    for (uint64_t i = start; i < n; i++) {
        uint32_t t = edge_to(m, s, text[i]);
        if (t == FAIL) break;
        s = t;
        if (k < cap) states[k] = s;
        k++;
    }
    return k;
}

int oracle_pfac(const oracle_machine *m, const uint8_t *text, uint64_t n,
                uint32_t **pairs, uint64_t *M) {
    pairbuf b = {0};
    for (uint64_t start = 0; start < n; start++) {
        uint32_t s = 0;
        for (uint64_t i = start; i < n; i++) {
            uint32_t t = edge_to(m, s, text[i]);
            if (t == FAIL) break;
            s = t;
            const ostate *q = &m->st[s];
            for (uint32_t k = 0; k < q->nown; k++) pb_push(&b, (uint32_t)i, q->own[k]);
        }
    }
    return finish(&b, pairs, M);
}

/* The definition of M, written out. */
int oracle_brute(const uint8_t *const *pats, const uint32_t *lens, uint32_t P,
                 const uint8_t *text, uint64_t n, uint32_t **pairs, uint64_t *M) {
    pairbuf b = {0};
    for (uint64_t e = 0; e < n; e++)
        for (uint32_t j = 0; j < P; j++) {
            uint64_t L = lens[j];
            if (L == 0 || L > e + 1) continue;
            if (memcmp(text + (e + 1 - L), pats[j], (size_t)L) == 0) pb_push(&b, (uint32_t)e, j);
        }
    return finish(&b, pairs, M);
}

/* counts[j] = number of matches of pattern j */
void oracle_counts(const uint32_t *pairs, uint64_t M, uint32_t P, uint64_t *counts) {
    memset(counts, 0, (size_t)P * sizeof(uint64_t));
    for (uint64_t i = 0; i < M; i++)
        if (pairs[2 * i + 1] < P) counts[pairs[2 * i + 1]]++;
}

void oracle_free_buf(void *p) { free(p); }
