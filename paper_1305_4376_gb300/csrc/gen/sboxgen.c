/*
 * sboxgen.c -- search for LOP3 (3-input lookup table) circuits that compute
 * the DES S-boxes S1..S8, for the bitsliced kernel.
 *
 * Every S-box maps 6 input bits b1..b6 to 4 output bits: the row is b1 b6,
 * the column b2 b3 b4 b5 (FIPS 46-3).  In the bitsliced kernel each bit is a
 * 32-bit word holding that bit of 32 different blocks, and a gate is one
 * lop3.b32 instruction, which can compute ANY boolean function of 3 words.
 * The number of gates is the kernel's arithmetic cost, so we search for
 * small circuits.
 *
 * Method (a recursive multiplexer decomposition with don't-cares, in the
 * spirit of Kwan's bitslice gate-count reduction, adapted to 3-input LUTs):
 *   solve(f on care set M):
 *     1. f already exists (or its complement) on M       -> 0 new gates
 *     2. f is a function of some 3 existing nodes on M    -> 1 gate
 *     3. f = LUT(g, a, b) with a, b existing and g a new
 *        gate of 3 existing nodes                          -> 2 gates
 *     4. pick an input bit s; solve f on M & ~s, then on M & s with the
 *        help of the first half's result (f itself, f ^ h0, or f restricted
 *        to where h0 decides it), join with one LUT(s, h0, h1); keep the
 *        cheapest choice of s and join.  Optionally, near the top of an
 *        output, s may also be any gate already built.
 *   The four outputs are solved one after another, each reusing every gate
 *   built so far; output orders and random tie-breaks are tried, and the
 *   smallest circuit wins.  Finally dead gates are removed and single-use
 *   gates are merged into their consumer whenever the pair still has at most
 *   three distinct inputs, and a gate is redefined on any three other nodes
 *   that compute the same function when that lets gates die
 *   (resubstitution).  Optionally a rip-up-and-reroute pass then takes
 *   out the gates only one output (or two) needs and solves those outputs
 *   again on top of the rest, keeping any strictly smaller result.
 *
 * Every circuit written out is verified exhaustively on all 64 inputs.
 * Negation is free: a consumer LUT absorbs it, so references carry a
 * complement flag.  Output: one JSON object per S-box on stdout.
 *
 * Build and run (offline; the result is committed):
 *   gcc -O2 -o sboxgen sboxgen.c
 *   ./sboxgen restarts seed step3_maxn var_depth step3_depth max_budget [sbox [improve [gate_sel [best.json]]]] > out.json
 *   ./sboxgen --polish in.json sbox seed seconds out.json
 * (the second form rebuilds fanout-free cones of an existing circuit from the
 * rest of it with fewer gates, and re-solves outputs, for a fixed time)
 * (merge_circuits.py keeps the smallest verified circuit per S-box over
 * several runs.)
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef uint64_t tt_t;

/* S-boxes of FIPS 46-3, 4 rows x 16 columns each. */
static const int SBOX[8][4][16] = {
    {{14, 4, 13, 1, 2, 15, 11, 8, 3, 10, 6, 12, 5, 9, 0, 7},
     {0, 15, 7, 4, 14, 2, 13, 1, 10, 6, 12, 11, 9, 5, 3, 8},
     {4, 1, 14, 8, 13, 6, 2, 11, 15, 12, 9, 7, 3, 10, 5, 0},
     {15, 12, 8, 2, 4, 9, 1, 7, 5, 11, 3, 14, 10, 0, 6, 13}},
    {{15, 1, 8, 14, 6, 11, 3, 4, 9, 7, 2, 13, 12, 0, 5, 10},
     {3, 13, 4, 7, 15, 2, 8, 14, 12, 0, 1, 10, 6, 9, 11, 5},
     {0, 14, 7, 11, 10, 4, 13, 1, 5, 8, 12, 6, 9, 3, 2, 15},
     {13, 8, 10, 1, 3, 15, 4, 2, 11, 6, 7, 12, 0, 5, 14, 9}},
    {{10, 0, 9, 14, 6, 3, 15, 5, 1, 13, 12, 7, 11, 4, 2, 8},
     {13, 7, 0, 9, 3, 4, 6, 10, 2, 8, 5, 14, 12, 11, 15, 1},
     {13, 6, 4, 9, 8, 15, 3, 0, 11, 1, 2, 12, 5, 10, 14, 7},
     {1, 10, 13, 0, 6, 9, 8, 7, 4, 15, 14, 3, 11, 5, 2, 12}},
    {{7, 13, 14, 3, 0, 6, 9, 10, 1, 2, 8, 5, 11, 12, 4, 15},
     {13, 8, 11, 5, 6, 15, 0, 3, 4, 7, 2, 12, 1, 10, 14, 9},
     {10, 6, 9, 0, 12, 11, 7, 13, 15, 1, 3, 14, 5, 2, 8, 4},
     {3, 15, 0, 6, 10, 1, 13, 8, 9, 4, 5, 11, 12, 7, 2, 14}},
    {{2, 12, 4, 1, 7, 10, 11, 6, 8, 5, 3, 15, 13, 0, 14, 9},
     {14, 11, 2, 12, 4, 7, 13, 1, 5, 0, 15, 10, 3, 9, 8, 6},
     {4, 2, 1, 11, 10, 13, 7, 8, 15, 9, 12, 5, 6, 3, 0, 14},
     {11, 8, 12, 7, 1, 14, 2, 13, 6, 15, 0, 9, 10, 4, 5, 3}},
    {{12, 1, 10, 15, 9, 2, 6, 8, 0, 13, 3, 4, 14, 7, 5, 11},
     {10, 15, 4, 2, 7, 12, 9, 5, 6, 1, 13, 14, 0, 11, 3, 8},
     {9, 14, 15, 5, 2, 8, 12, 3, 7, 0, 4, 10, 1, 13, 11, 6},
     {4, 3, 2, 12, 9, 5, 15, 10, 11, 14, 1, 7, 6, 0, 8, 13}},
    {{4, 11, 2, 14, 15, 0, 8, 13, 3, 12, 9, 7, 5, 10, 6, 1},
     {13, 0, 11, 7, 4, 9, 1, 10, 14, 3, 5, 12, 2, 15, 8, 6},
     {1, 4, 11, 13, 12, 3, 7, 14, 10, 15, 6, 8, 0, 5, 9, 2},
     {6, 11, 13, 8, 1, 4, 10, 7, 9, 5, 0, 15, 14, 2, 3, 12}},
    {{13, 2, 8, 4, 6, 15, 11, 1, 10, 9, 3, 14, 5, 0, 12, 7},
     {1, 15, 13, 8, 10, 3, 7, 4, 12, 5, 6, 11, 0, 14, 9, 2},
     {7, 11, 4, 1, 9, 12, 14, 2, 0, 6, 10, 13, 15, 3, 5, 8},
     {2, 1, 14, 7, 4, 10, 8, 13, 15, 12, 9, 0, 3, 5, 6, 11}}};

#define MAXN 96
#define ALL (~(tt_t)0)

typedef struct {
    int n;                 /* nodes 0..5 are the inputs b1..b6 */
    tt_t tt[MAXN];
    int in[MAXN][3];       /* gate inputs (node ids) */
    uint8_t imm[MAXN];     /* lop3 truth table: bit (4a+2b+c) */
} state_t;

/* search knobs */
static int g_use_step3 = 1;
static int g_step3_maxn = 40;
static int g_variants = 1;
static int g_max_budget = 16;
static int g_var_depth = 1;   /* join variants explored above this depth */
static int g_two_depth = 1;   /* step 3 used above this depth */
static int g_improve_rounds = 0; /* rip-up-and-reroute attempts per circuit */
static int g_node_sel = 0;       /* also split on existing gates above this depth (1 = top only) */
static const char* g_best_path = NULL; /* with a single S-box: rewrite this file on every improvement */
static uint64_t g_rng = 88172645463325252ull;

static uint64_t rnd(void) {
    g_rng ^= g_rng << 13;
    g_rng ^= g_rng >> 7;
    g_rng ^= g_rng << 17;
    return g_rng;
}

static tt_t input_tt(int m) { /* b_{m+1}: bit (5-m) of the point index */
    tt_t t = 0;
    for (int p = 0; p < 64; p++)
        if ((p >> (5 - m)) & 1) t |= (tt_t)1 << p;
    return t;
}

static tt_t eval_lut(tt_t a, tt_t b, tt_t c, uint8_t imm) {
    tt_t r = 0;
    for (int k = 0; k < 8; k++)
        if ((imm >> k) & 1) r |= ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c);
    return r;
}

/* Is target (on mask) a function of (a, b, c)?  Returns imm or -1.
 * Combinations that never occur on the mask are don't-cares, filled from
 * `fill` so that restarts explore different completions. */
static int lut_fit(tt_t a, tt_t b, tt_t c, tt_t target, tt_t mask, uint8_t fill) {
    int imm = 0;
    for (int k = 0; k < 8; k++) {
        tt_t sel = ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c) & mask;
        if (sel & target) {
            if (sel & ~target) return -1;
            imm |= 1 << k;
        } else if (!sel) {
            imm |= fill & (1 << k);
        }
    }
    return imm;
}

static int add_gate(state_t* s, int a, int b, int c, int imm) {
    int n = s->n++;
    s->in[n][0] = a;
    s->in[n][1] = b;
    s->in[n][2] = c;
    s->imm[n] = (uint8_t)imm;
    s->tt[n] = eval_lut(s->tt[a], s->tt[b], s->tt[c], (uint8_t)imm);
    return n;
}

/* references: node*2 + complement */
static int find_existing(const state_t* s, tt_t target, tt_t mask) {
    for (int i = 0; i < s->n; i++) {
        tt_t d = (s->tt[i] ^ target) & mask;
        if (d == 0) return 2 * i;
        if (d == mask) return 2 * i + 1;
    }
    return -1;
}

static tt_t ref_tt(const state_t* s, int r) { return (r & 1) ? ~s->tt[r >> 1] : s->tt[r >> 1]; }

static int find_triple(const state_t* s, tt_t target, tt_t mask, int* oi, int* oj, int* ok, int* oimm) {
    int n = s->n;
    int off = (int)(rnd() % (uint64_t)n);
    uint8_t fill = (uint8_t)rnd();
    for (int ii = 0; ii < n; ii++) {
        int i = (ii + off) % n;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            for (int k = j + 1; k < n; k++) {
                if (k == i) continue;
                int imm = lut_fit(s->tt[i], s->tt[j], s->tt[k], target, mask, fill);
                if (imm >= 0) {
                    *oi = i; *oj = j; *ok = k; *oimm = imm;
                    return 1;
                }
            }
        }
    }
    return 0;
}

/* Step 3: target = LUT(g, a, b), g = LUT of three existing nodes. */
static int find_two(state_t* s, tt_t target, tt_t mask) {
    int n = s->n;
    if (n > g_step3_maxn) return -1;
    for (int a = 0; a < n; a++) {
        for (int b = a; b < n; b++) {
            tt_t ta = s->tt[a], tb = s->tt[b];
            tt_t cls[4];
            cls[0] = ~ta & ~tb & mask; cls[1] = ~ta & tb & mask;
            cls[2] = ta & ~tb & mask;  cls[3] = ta & tb & mask;
            int var[4], nv = 0;
            tt_t fixed_care = 0;
            for (int q = 0; q < 4; q++) {
                if (!cls[q]) continue;
                if ((cls[q] & target) && (cls[q] & ~target)) var[nv++] = q;
                else fixed_care |= cls[q];
            }
            (void)fixed_care;
            if (nv == 0) continue; /* then step 2 would have found it */
            for (int pol = 0; pol < (1 << nv); pol++) {
                tt_t req = 0, rmask = 0;
                for (int v = 0; v < nv; v++) {
                    tt_t c = cls[var[v]];
                    rmask |= c;
                    req |= ((pol >> v) & 1) ? (~target & c) : (target & c);
                }
                int i, j, k, imm;
                if (find_triple(s, req, rmask, &i, &j, &k, &imm)) {
                    int g = add_gate(s, i, j, k, imm);
                    int imm2 = lut_fit(s->tt[g], ta, tb, target, mask, (uint8_t)rnd());
                    if (imm2 < 0) { s->n--; continue; }
                    int f = add_gate(s, g, a, b, imm2);
                    return 2 * f;
                }
            }
        }
    }
    return -1;
}

static int solve(state_t* s, tt_t target, tt_t mask, int used, int budget);
/* inputs used as selectors are bits 0..5; gate selectors are counted from bit 8 */
static int depth_of(int used) { return __builtin_popcount(used & 63) + (used >> 8); }

/* Step 4: decomposition on input bit `sel`, `first` = which half first. */
static int split(state_t* s, tt_t target, tt_t mask, int used, int sel, int first, int budget) {
    tt_t xs = s->tt[sel];
    tt_t m0 = mask & (first ? xs : ~xs);
    tt_t m1 = mask & ~m0;
    if (!m0 || !m1) return -1;
    state_t base = *s;
    /* an input selector is not used again below; a gate selector (only at
     * the top of an output) counts as one level of depth */
    const int nused = sel < 6 ? used | (1 << sel) : used + (1 << 8);
    int r0 = solve(&base, target, m0, nused, budget - 1);
    if (r0 < 0) return -1;
    int spent0 = base.n - s->n;
    if (spent0 + 1 > budget) return -1;
    tt_t t0 = ref_tt(&base, r0);
    tt_t f1 = target & m1;
    /* candidate requirements for the second half */
    tt_t req[6], rm[6];
    int nreq = 0;
    req[nreq] = target; rm[nreq++] = m1;
    if (g_variants && depth_of(used) < g_var_depth) {
        req[nreq] = target ^ t0; rm[nreq++] = m1;
        if ((f1 & ~t0) == 0) { req[nreq] = target; rm[nreq++] = m1 & t0; }          /* f = t0 & h */
        if (((~target & m1) & t0) == 0) { req[nreq] = target; rm[nreq++] = m1 & ~t0; } /* f = t0 | h */
        if ((f1 & t0) == 0) { req[nreq] = target; rm[nreq++] = m1 & ~t0; }          /* f = ~t0 & h */
        if (((~target & m1) & ~t0) == 0) { req[nreq] = target; rm[nreq++] = m1 & t0; } /* f = ~t0 | h */
    }
    int best = -1;
    state_t best_s;
    for (int v = 0; v < nreq; v++) {
        int b = (best >= 0 ? (best_s.n - s->n) - 1 : budget) - spent0 - 1;
        if (b < 0) break;
        state_t c = base;
        int r1;
        if (rm[v] == 0) {
            r1 = r0; /* second half free: any node works, reuse */
        } else {
            r1 = solve(&c, req[v], rm[v], nused, b);
        }
        if (r1 < 0) continue;
        int a1 = r0 >> 1, b1 = r1 >> 1;
        int imm = lut_fit(xs, c.tt[a1], c.tt[b1], target, mask, (uint8_t)rnd());
        if (imm < 0) continue;
        int g = add_gate(&c, sel, a1, b1, imm);
        if (best < 0 || c.n < best_s.n) {
            best = 2 * g;
            best_s = c;
        }
    }
    if (best >= 0) *s = best_s;
    return best;
}

static int solve(state_t* s, tt_t target, tt_t mask, int used, int budget) {
    int r = find_existing(s, target, mask);
    if (r >= 0) return r;
    if (budget < 1 || s->n + 1 >= MAXN) return -1;
    int i, j, k, imm;
    if (find_triple(s, target, mask, &i, &j, &k, &imm)) return 2 * add_gate(s, i, j, k, imm);
    if (budget < 2 || s->n + 2 >= MAXN) return -1;
    if (g_use_step3 && depth_of(used) < g_two_depth) {
        state_t c = *s;
        r = find_two(&c, target, mask);
        if (r >= 0) {
            *s = c;
            return r;
        }
    }
    if (budget < 3) return -1;
    int best = -1;
    state_t best_s;
    int order[6];
    for (int q = 0; q < 6; q++) order[q] = q;
    for (int q = 5; q > 0; q--) {
        int t = (int)(rnd() % (uint64_t)(q + 1));
        int x = order[q]; order[q] = order[t]; order[t] = x;
    }
    for (int qi = 0; qi < 6; qi++) {
        int sel = order[qi];
        if (used & (1 << sel)) continue;
        for (int first = 0; first < 2; first++) {
            int b = best >= 0 ? (best_s.n - s->n) - 1 : budget;
            if (b < 3) break;
            state_t c = *s;
            int rr = split(&c, target, mask, used, sel, first, b);
            if (rr >= 0 && (best < 0 || c.n < best_s.n)) {
                best = rr;
                best_s = c;
            }
        }
    }
    /* gates as selectors: f = LUT(g, h0, h1) split on an existing gate g */
    if (g_node_sel && depth_of(used) < g_node_sel) {
        for (int g = 6; g < s->n; g++) {
            for (int first = 0; first < 2; first++) {
                int b = best >= 0 ? (best_s.n - s->n) - 1 : budget;
                if (b < 3) break;
                state_t c = *s;
                int rr = split(&c, target, mask, used, g, first, b);
                if (rr >= 0 && (best < 0 || c.n < best_s.n)) {
                    best = rr;
                    best_s = c;
                }
            }
        }
    }
    if (best >= 0) *s = best_s;
    return best;
}

/* ---- post-passes ---- */

static void remove_dead(state_t* s, int outs[4]) {
    int live[MAXN] = {0};
    for (int t = 0; t < 4; t++) live[outs[t] >> 1] = 1;
    for (int n = s->n - 1; n >= 6; n--)
        if (live[n])
            for (int q = 0; q < 3; q++) live[s->in[n][q]] = 1;
    int map[MAXN];
    state_t d = *s;
    d.n = 6;
    for (int n = 0; n < 6; n++) map[n] = n;
    for (int n = 6; n < s->n; n++) {
        if (!live[n]) continue;
        int m = d.n++;
        map[n] = m;
        for (int q = 0; q < 3; q++) d.in[m][q] = map[s->in[n][q]];
        d.imm[m] = s->imm[n];
        d.tt[m] = s->tt[n];
    }
    for (int t = 0; t < 4; t++) outs[t] = 2 * map[outs[t] >> 1] + (outs[t] & 1);
    *s = d;
}

/* Merge gate g into its only consumer h when inputs(g) U inputs(h)\{g} has at
 * most 3 distinct nodes and g is not an output. */
static int merge_pass(state_t* s, int outs[4]) {
    int changed = 0;
    for (int g = 6; g < s->n; g++) {
        int uses = 0, user = -1;
        for (int h = g + 1; h < s->n; h++)
            for (int q = 0; q < 3; q++)
                if (s->in[h][q] == g) { uses++; user = h; }
        int is_out = 0;
        for (int t = 0; t < 4; t++) if ((outs[t] >> 1) == g) is_out = 1;
        if (uses == 0 || is_out) continue;
        /* count distinct inputs of user, counting each occurrence once */
        int set[6], ns = 0;
        for (int q = 0; q < 3; q++) {
            int x = s->in[g][q], dup = 0;
            for (int z = 0; z < ns; z++) if (set[z] == x) dup = 1;
            if (!dup) set[ns++] = x;
        }
        for (int q = 0; q < 3; q++) {
            int x = s->in[user][q], dup = 0;
            if (x == g) continue;
            for (int z = 0; z < ns; z++) if (set[z] == x) dup = 1;
            if (!dup) set[ns++] = x;
        }
        if (uses != 1 || ns > 3) continue;
        while (ns < 3) set[ns++] = set[0];
        int imm = lut_fit(s->tt[set[0]], s->tt[set[1]], s->tt[set[2]], s->tt[user], ALL, 0);
        if (imm < 0) continue;
        s->in[user][0] = set[0]; s->in[user][1] = set[1]; s->in[user][2] = set[2];
        s->imm[user] = (uint8_t)imm;
        /* g is now dead; drop it */
        remove_dead(s, outs);
        changed = 1;
        g = 5;
    }
    return changed;
}

/* Renumbers the nodes in a topological order (inputs first); returns 0 if
 * the gate list has a cycle. */
static int toposort(state_t* s, int outs[4]) {
    int order[MAXN], pos[MAXN], done[MAXN] = {0}, no = 0;
    for (int m = 0; m < 6; m++) { order[no++] = m; done[m] = 1; }
    while (no < s->n) {
        int progress = 0;
        for (int n = 6; n < s->n; n++) {
            if (done[n]) continue;
            if (done[s->in[n][0]] && done[s->in[n][1]] && done[s->in[n][2]]) {
                order[no++] = n;
                done[n] = 1;
                progress = 1;
            }
        }
        if (!progress) return 0;
    }
    for (int i = 0; i < s->n; i++) pos[order[i]] = i;
    state_t d = *s;
    for (int i = 6; i < s->n; i++) {
        const int o = order[i];
        for (int q = 0; q < 3; q++) d.in[i][q] = pos[s->in[o][q]];
        d.imm[i] = s->imm[o];
        d.tt[i] = s->tt[o];
    }
    for (int t = 0; t < 4; t++) outs[t] = 2 * pos[outs[t] >> 1] + (outs[t] & 1);
    *s = d;
    return 1;
}

/* Resubstitution: a gate whose function is also a LUT of three other nodes
 * outside its transitive fanout is redefined on them; whatever no longer
 * feeds an output is removed.  Kept only when the circuit gets smaller. */
static int resub_pass(state_t* s, int outs[4]) {
    int improved = 0;
    for (int g = 6; g < s->n; g++) {
        char tfo[MAXN] = {0};
        tfo[g] = 1;
        for (int n = g + 1; n < s->n; n++)
            if (tfo[s->in[n][0]] || tfo[s->in[n][1]] || tfo[s->in[n][2]]) tfo[n] = 1;
        int cand[MAXN], nc = 0;
        for (int n = 0; n < s->n; n++)
            if (!tfo[n]) cand[nc++] = n;
        int done = 0;
        for (int i = 0; i < nc && !done; i++)
            for (int j = i; j < nc && !done; j++)
                for (int k = j; k < nc && !done; k++) {
                    const int a = cand[i], b = cand[j], c = cand[k];
                    const int imm = lut_fit(s->tt[a], s->tt[b], s->tt[c], s->tt[g], ALL, 0);
                    if (imm < 0) continue;
                    if (a == s->in[g][0] && b == s->in[g][1] && c == s->in[g][2]) continue;
                    state_t t = *s;
                    int to[4];
                    memcpy(to, outs, sizeof(to));
                    t.in[g][0] = a; t.in[g][1] = b; t.in[g][2] = c;
                    t.imm[g] = (uint8_t)imm;
                    if (!toposort(&t, to)) continue;
                    remove_dead(&t, to);
                    if (t.n < s->n) {
                        *s = t;
                        memcpy(outs, to, sizeof(to));
                        improved = 1;
                        done = 1;
                        g = 5; /* indices changed: start over */
                    }
                }
    }
    return improved;
}

static int verify(const state_t* s, const int outs[4], int box) {
    for (int p = 0; p < 64; p++) {
        int row = ((p >> 5) & 1) * 2 + (p & 1), col = (p >> 1) & 15;
        int v = SBOX[box][row][col];
        /* re-evaluate the circuit from its gate list, not the cached tables */
        int val[MAXN];
        for (int m = 0; m < 6; m++) val[m] = (p >> (5 - m)) & 1;
        for (int n = 6; n < s->n; n++) {
            int k = val[s->in[n][0]] * 4 + val[s->in[n][1]] * 2 + val[s->in[n][2]];
            val[n] = (s->imm[n] >> k) & 1;
        }
        for (int t = 0; t < 4; t++) {
            int bit = val[outs[t] >> 1] ^ (outs[t] & 1);
            if (bit != ((v >> (3 - t)) & 1)) return 0;
        }
    }
    return 1;
}

/* Rip-up and reroute: take the gates only output t (or outputs t and u)
 * needs out of the circuit, and solve those outputs again, cheapest budget
 * first, with everything else kept; accept only a strictly smaller circuit. */
static int cone_exclusive(const state_t* s, const int outs[4], int drop_mask, int* cnt) {
    int keep[MAXN] = {0}, need[MAXN] = {0};
    for (int t = 0; t < 4; t++) {
        int* mark = (drop_mask >> t) & 1 ? need : keep;
        mark[outs[t] >> 1] = 1;
    }
    for (int n = s->n - 1; n >= 6; n--) {
        if (keep[n]) for (int q = 0; q < 3; q++) keep[s->in[n][q]] = 1;
        if (need[n]) for (int q = 0; q < 3; q++) need[s->in[n][q]] = 1;
    }
    int c = 0;
    for (int n = 6; n < s->n; n++) if (need[n] && !keep[n]) c++;
    *cnt = c;
    return c;
}

static int improve_once(state_t* s, int outs[4], tt_t targets[4], int drop_mask) {
    int excl = 0;
    cone_exclusive(s, outs, drop_mask, &excl);
    if (excl < 2) return 0;
    state_t base = *s;
    int bo[4];
    memcpy(bo, outs, sizeof(bo));
    for (int t = 0; t < 4; t++) if ((drop_mask >> t) & 1) bo[t] = 0; /* park on an input */
    remove_dead(&base, bo);
    const int base_gates = base.n - 6;
    const int old_gates = s->n - 6;
    int order[4], no = 0;
    for (int t = 0; t < 4; t++) if ((drop_mask >> t) & 1) order[no++] = t;
    if (no == 2 && (rnd() & 1)) { int x = order[0]; order[0] = order[1]; order[1] = x; }
    state_t cur = base;
    for (int i = 0; i < no; i++) {
        const int t = order[i];
        const int room = old_gates - 1 - (cur.n - 6);
        int r = -1;
        for (int lim = 0; lim <= room && r < 0; lim++) {
            state_t c = cur;
            r = solve(&c, targets[t], ALL, 0, lim);
            if (r >= 0) cur = c;
        }
        if (r < 0) return 0;
        bo[t] = r;
    }
    remove_dead(&cur, bo);
    while (merge_pass(&cur, bo)) {}
    (void)base_gates;
    if (cur.n - 6 < old_gates) {
        *s = cur;
        memcpy(outs, bo, sizeof(bo));
        return 1;
    }
    return 0;
}

static void improve(state_t* s, int outs[4], tt_t targets[4], int rounds) {
    for (int it = 0; it < rounds; it++) {
        int mask = (int)(rnd() % 10);
        /* single outputs and pairs */
        static const int masks[10] = {1, 2, 4, 8, 3, 5, 9, 6, 10, 12};
        improve_once(s, outs, targets, masks[mask]);
    }
}

/* ---- polish mode: windowed resynthesis of an existing circuit ----
 *
 * For a gate r, its maximum fanout-free cone (MFFC) is r together with every
 * gate all of whose consumers lie in the cone (outputs other than r excluded):
 * the gates that die when r is computed some other way.  polish_once() picks
 * r at random, keeps every node outside the MFFC that does not depend on r,
 * and asks the recursive solver for tt[r] from those nodes with fewer new
 * gates than the cone had; the gates that read r are then rewired to the new
 * node.  Outputs that are themselves such roots may come back complemented. */

static int mffc_of(const state_t* s, const int outs[4], int r, char* in_cone) {
    memset(in_cone, 0, MAXN);
    in_cone[r] = 1;
    int size = 1, changed = 1;
    while (changed) {
        changed = 0;
        for (int n = r - 1; n >= 6; n--) {
            if (in_cone[n]) continue;
            int is_out = 0;
            for (int t = 0; t < 4; t++) if ((outs[t] >> 1) == n) is_out = 1;
            if (is_out) continue;
            int uses = 0, inside = 1;
            for (int h = n + 1; h < s->n; h++)
                for (int q = 0; q < 3; q++)
                    if (s->in[h][q] == n) {
                        uses++;
                        if (!in_cone[h]) inside = 0;
                    }
            if (uses && inside) {
                in_cone[n] = 1;
                size++;
                changed = 1;
            }
        }
    }
    return size;
}

static int polish_once(state_t* s, int outs[4], int box) {
    if (s->n <= 7) return 0;
    const int r = 6 + (int)(rnd() % (uint64_t)(s->n - 6));
    char cone[MAXN], tfo[MAXN] = {0};
    const int m = mffc_of(s, outs, r, cone);
    if (m < 2) return 0;
    for (int n = r + 1; n < s->n; n++)
        if (tfo[s->in[n][0]] || tfo[s->in[n][1]] || tfo[s->in[n][2]] ||
            s->in[n][0] == r || s->in[n][1] == r || s->in[n][2] == r)
            tfo[n] = 1;
    /* base: the nodes outside the cone that do not depend on r */
    state_t b;
    int map[MAXN];
    b.n = 6;
    for (int q = 0; q < 6; q++) { b.tt[q] = s->tt[q]; map[q] = q; }
    for (int n = 6; n < s->n; n++) {
        map[n] = -1;
        if (cone[n] || tfo[n]) continue;
        const int k = b.n++;
        for (int q = 0; q < 3; q++) b.in[k][q] = map[s->in[n][q]];
        b.imm[k] = s->imm[n];
        b.tt[k] = s->tt[n];
        map[n] = k;
    }
    /* rebuild tt[r] with at most m - 1 new gates, cheapest first */
    int ref = -1;
    state_t c;
    for (int lim = 0; lim < m && ref < 0; lim++) {
        c = b;
        ref = solve(&c, s->tt[r], ALL, 0, lim);
    }
    if (ref < 0) return 0;
    if (ref & 1) { /* complemented: only an output may take it as it is */
        int ok = 1;
        for (int n = r + 1; n < s->n; n++)
            if (tfo[n] && (s->in[n][0] == r || s->in[n][1] == r || s->in[n][2] == r)) ok = 0;
        if (!ok) return 0;
    }
    /* append the gates that depend on r, reading the new node instead */
    for (int n = r + 1; n < s->n; n++) {
        if (!tfo[n]) continue;
        const int k = c.n++;
        uint8_t imm = s->imm[n];
        for (int q = 0; q < 3; q++) c.in[k][q] = s->in[n][q] == r ? ref >> 1 : map[s->in[n][q]];
        c.imm[k] = imm;
        c.tt[k] = eval_lut(c.tt[c.in[k][0]], c.tt[c.in[k][1]], c.tt[c.in[k][2]], imm);
        map[n] = k;
    }
    int no[4];
    for (int t = 0; t < 4; t++) {
        const int o = outs[t] >> 1;
        no[t] = o == r ? (ref ^ (outs[t] & 1)) : 2 * map[o] + (outs[t] & 1);
        if ((o != r) && map[o] < 0) return 0;
    }
    remove_dead(&c, no);
    while (merge_pass(&c, no)) {}
    if (c.n >= s->n || !verify(&c, no, box)) return 0;
    *s = c;
    memcpy(outs, no, sizeof(no));
    return 1;
}

/* minimal reader of {"sbox": k, "gates": [[a,b,c,imm],...], "outputs": [...]} */
static int read_num(const char** p, const char* end) {
    while (*p < end && !(**p >= '0' && **p <= '9')) (*p)++;
    int v = 0;
    while (*p < end && **p >= '0' && **p <= '9') v = v * 10 + (*(*p)++ - '0');
    return v;
}

static int load_circuit(const char* path, int box, state_t* s, int outs[4]) {
    FILE* f = fopen(path, "rb");
    if (!f) return 0;
    static char buf[1 << 20];
    size_t len = fread(buf, 1, sizeof(buf) - 1, f);
    fclose(f);
    buf[len] = 0;
    for (const char* p = buf; (p = strstr(p, "\"sbox\"")) != NULL;) {
        const char* q = p + 6;
        const int k = read_num(&q, buf + len);
        const char* gs = strstr(q, "\"gates\"");
        const char* os = gs ? strstr(gs, "\"outputs\"") : NULL;
        if (!gs || !os) return 0;
        const char* nx = strstr(os, "\"sbox\"");
        if (k == box + 1) {
            s->n = 6;
            for (int m = 0; m < 6; m++) s->tt[m] = input_tt(m);
            const char* r = gs + 7;
            for (;;) {
                const char* t = r;
                while (t < os && !(*t >= '0' && *t <= '9')) t++;
                if (t >= os || s->n + 1 >= MAXN) break;
                int a = read_num(&r, os), b2 = read_num(&r, os), c = read_num(&r, os), imm = read_num(&r, os);
                if (a >= s->n || b2 >= s->n || c >= s->n) return 0;
                add_gate(s, a, b2, c, imm);
            }
            r = os + 9;
            for (int t = 0; t < 4; t++) outs[t] = read_num(&r, nx ? nx : buf + len);
            return verify(s, outs, box);
        }
        p = nx ? nx : buf + len;
        if (!nx) break;
    }
    return 0;
}

static void write_circuit(const char* path, const state_t* s, const int outs[4], int box) {
    char tmp[4096];
    snprintf(tmp, sizeof tmp, "%s.tmp", path);
    FILE* f = fopen(tmp, "w");
    if (!f) return;
    fprintf(f, "[{\"sbox\": %d, \"gates\": [", box + 1);
    for (int n = 6; n < s->n; n++)
        fprintf(f, "%s[%d, %d, %d, %d]", n > 6 ? ", " : "", s->in[n][0], s->in[n][1], s->in[n][2], s->imm[n]);
    fprintf(f, "], \"outputs\": [%d, %d, %d, %d]}]\n", outs[0], outs[1], outs[2], outs[3]);
    fclose(f);
    rename(tmp, path);
}

/* sboxgen --polish in.json sbox seed seconds out.json: windowed resynthesis
 * and rip-up-and-reroute of the circuit for one S-box, for a fixed time. */
static int polish_main(int argc, char** argv) {
    if (argc < 7) {
        fprintf(stderr, "usage: %s --polish in.json sbox seed seconds out.json\n", argv[0]);
        return 2;
    }
    const int box = atoi(argv[3]) - 1;
    if (box < 0 || box > 7) return 2;
    g_rng ^= strtoull(argv[4], NULL, 0) * 0x9E3779B97F4A7C15ull;
    const double seconds = atof(argv[5]);
    state_t s;
    int outs[4];
    if (!load_circuit(argv[2], box, &s, outs)) {
        fprintf(stderr, "no valid circuit for S%d in %s\n", box + 1, argv[2]);
        return 1;
    }
    tt_t targets[4];
    for (int t = 0; t < 4; t++) {
        targets[t] = 0;
        for (int p = 0; p < 64; p++) {
            int row = ((p >> 5) & 1) * 2 + (p & 1), col = (p >> 1) & 15;
            if ((SBOX[box][row][col] >> (3 - t)) & 1) targets[t] |= (tt_t)1 << p;
        }
    }
    fprintf(stderr, "S%d: start %d gates\n", box + 1, s.n - 6);
    const clock_t t0 = clock();
    long tries = 0;
    while ((double)(clock() - t0) / CLOCKS_PER_SEC < seconds) {
        const int before = s.n;
        if (rnd() % 4) polish_once(&s, outs, box);
        else improve(&s, outs, targets, 1);
        while (merge_pass(&s, outs) || resub_pass(&s, outs)) {}
        tries++;
        if (s.n < before) {
            if (!verify(&s, outs, box)) {
                fprintf(stderr, "internal error: polished circuit for S%d fails verification\n", box + 1);
                return 1;
            }
            write_circuit(argv[6], &s, outs, box);
            fprintf(stderr, "S%d: %d gates (try %ld)\n", box + 1, s.n - 6, tries);
        }
    }
    fprintf(stderr, "S%d: done, %d gates after %ld tries\n", box + 1, s.n - 6, tries);
    return 0;
}

int main(int argc, char** argv) {
    if (argc > 1 && strcmp(argv[1], "--polish") == 0) return polish_main(argc, argv);
    int restarts = argc > 1 ? atoi(argv[1]) : 20;
    g_rng ^= argc > 2 ? strtoull(argv[2], NULL, 0) * 0x9E3779B97F4A7C15ull : 0;
    if (argc > 3) g_step3_maxn = atoi(argv[3]);
    if (argc > 4) g_var_depth = atoi(argv[4]);
    if (argc > 5) g_two_depth = atoi(argv[5]);
    if (argc > 6) g_max_budget = atoi(argv[6]);
    const int only = argc > 7 ? atoi(argv[7]) : 0; /* 1..8: search this S-box only */
    if (argc > 8) g_improve_rounds = atoi(argv[8]);
    if (argc > 9) g_node_sel = atoi(argv[9]);
    if (argc > 10 && only) g_best_path = argv[10];
    tt_t targets[8][4];
    for (int box = 0; box < 8; box++)
        for (int t = 0; t < 4; t++) {
            tt_t v = 0;
            for (int p = 0; p < 64; p++) {
                int row = ((p >> 5) & 1) * 2 + (p & 1), col = (p >> 1) & 15;
                if ((SBOX[box][row][col] >> (3 - t)) & 1) v |= (tt_t)1 << p;
            }
            targets[box][t] = v;
        }
    static const int perms[24][4] = {
        {0,1,2,3},{0,1,3,2},{0,2,1,3},{0,2,3,1},{0,3,1,2},{0,3,2,1},
        {1,0,2,3},{1,0,3,2},{1,2,0,3},{1,2,3,0},{1,3,0,2},{1,3,2,0},
        {2,0,1,3},{2,0,3,1},{2,1,0,3},{2,1,3,0},{2,3,0,1},{2,3,1,0},
        {3,0,1,2},{3,0,2,1},{3,1,0,2},{3,1,2,0},{3,2,0,1},{3,2,1,0}};
    printf("[\n");
    int total = 0;
    int printed = 0;
    for (int box = 0; box < 8; box++) {
        if (only && box != only - 1) continue;
        state_t best;
        best.n = 6;
        int best_outs[4] = {0, 0, 0, 0}, best_n = 1 << 30;
        for (int rs = 0; rs < restarts; rs++) {
            for (int pi = 0; pi < 24; pi++) {
                state_t s;
                s.n = 6;
                for (int m = 0; m < 6; m++) s.tt[m] = input_tt(m);
                int outs[4], ok = 1;
                for (int q = 0; q < 4 && ok; q++) {
                    int t = perms[pi][q];
                    /* iterative deepening: the cheapest budget that works */
                    int r = -1;
                    for (int lim = 0; lim <= g_max_budget && r < 0; lim++) {
                        state_t c = s;
                        r = solve(&c, targets[box][t], ALL, 0, lim);
                        if (r >= 0) s = c;
                    }
                    if (r < 0) ok = 0;
                    else outs[t] = r;
                }
                if (!ok) continue;
                remove_dead(&s, outs);
                while (merge_pass(&s, outs) || resub_pass(&s, outs)) {}
                if (g_improve_rounds) improve(&s, outs, targets[box], g_improve_rounds);
                if (!verify(&s, outs, box)) {
                    fprintf(stderr, "internal error: circuit for S%d fails verification\n", box + 1);
                    return 1;
                }
                if (s.n - 6 < best_n) {
                    best_n = s.n - 6;
                    best = s;
                    memcpy(best_outs, outs, sizeof(outs));
                    fprintf(stderr, "S%d: %d gates (restart %d, order %d)\n", box + 1, best_n, rs, pi);
                    if (g_best_path) { /* keep the best circuit so far on disk */
                        FILE* f = fopen(g_best_path, "w");
                        if (f) {
                            fprintf(f, "[{\"sbox\": %d, \"gates\": [", box + 1);
                            for (int n = 6; n < best.n; n++)
                                fprintf(f, "%s[%d, %d, %d, %d]", n > 6 ? ", " : "", best.in[n][0], best.in[n][1],
                                        best.in[n][2], best.imm[n]);
                            fprintf(f, "], \"outputs\": [%d, %d, %d, %d]}]\n", best_outs[0], best_outs[1],
                                    best_outs[2], best_outs[3]);
                            fclose(f);
                        }
                    }
                }
            }
        }
        total += best_n;
        printf("%s {\"sbox\": %d, \"gates\": [", printed++ ? ",\n" : "", box + 1);
        for (int n = 6; n < best.n; n++)
            printf("%s[%d, %d, %d, %d]", n > 6 ? ", " : "", best.in[n][0], best.in[n][1], best.in[n][2], best.imm[n]);
        printf("], \"outputs\": [%d, %d, %d, %d]}", best_outs[0], best_outs[1], best_outs[2], best_outs[3]);
        fflush(stdout);
    }
    printf("\n]\n");
    fprintf(stderr, "total %d gates, mean %.2f per S-box\n", total, total / 8.0);
    return 0;
}
