/*
 * cgpopt.c -- shrink verified LOP3 circuits for the DES S-boxes by
 * Cartesian genetic programming (Miller's CGP, used as a circuit optimiser
 * under a correctness constraint in the manner of Vasicek and Sekanina).
 *
 * A circuit is a feed-forward list of 3-input lookup-table gates over the
 * S-box inputs b1..b6 (node ids 0..5) plus four output references
 * (node*2 + complement), the format sboxgen writes.  The optimiser keeps a
 * genome with a few spare gates beyond the ones in use, evaluates all gates
 * on the 64 input points as 64-bit truth tables, and runs a (1 + lambda)
 * evolution strategy:
 *   - each offspring changes a few genes: a gate input (any earlier node),
 *     a gate function, or an output reference;
 *   - an input change either keeps the gate's truth table when some function
 *     of the new inputs reproduces it (a neutral rewiring), or takes a random
 *     function;
 *   - an offspring is accepted only when all four outputs are still exact on
 *     all 64 points and it uses no more gates than its parent (ties are
 *     accepted, so the search drifts across equally small circuits); with a
 *     slack s > 0, one in ~4000 may also use up to s gates more than the
 *     best circuit so far.
 * The smallest circuit seen is written out whenever it improves.  It is
 * re-verified against the S-box table before every write.
 *
 *   gcc -O2 -o cgpopt cgpopt.c
 *   ./cgpopt in.json sbox seed seconds spare out.json [slack [drift.json]]
 * in.json holds one object per S-box (sboxgen's output or the committed
 * sbox_circuits.json); the circuit for `sbox` (1..8) is the start point.
 * merge_circuits.py then keeps the smallest verified circuit per S-box.
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

#define MAXG 80
#define NIN 6

typedef struct {
    int n;                   /* gates; node 6 + i is gate i */
    uint8_t in[MAXG][3];
    uint8_t imm[MAXG];
    int out[4];              /* node*2 + complement */
} geno_t;

static uint64_t g_rng = 0x9E3779B97F4A7C15ull;
static uint64_t rnd(void) {
    g_rng ^= g_rng << 13;
    g_rng ^= g_rng >> 7;
    g_rng ^= g_rng << 17;
    return g_rng;
}
static int rndn(int n) { return (int)(rnd() % (uint64_t)n); }

static tt_t g_in_tt[NIN];
static tt_t g_target[4];

static tt_t eval_lut(tt_t a, tt_t b, tt_t c, uint8_t imm) {
    tt_t r = 0;
    for (int k = 0; k < 8; k++)
        if ((imm >> k) & 1) r |= ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c);
    return r;
}

/* the function of (a, b, c) equal to target on all 64 points, or -1;
 * input combinations that never occur take random values */
static int lut_fit(tt_t a, tt_t b, tt_t c, tt_t target) {
    int imm = 0;
    uint8_t fill = (uint8_t)rnd();
    for (int k = 0; k < 8; k++) {
        tt_t sel = ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c);
        if (sel & target) {
            if (sel & ~target) return -1;
            imm |= 1 << k;
        } else if (!sel) {
            imm |= fill & (1 << k);
        }
    }
    return imm;
}

static void eval_all(const geno_t* g, tt_t* tt) {
    for (int m = 0; m < NIN; m++) tt[m] = g_in_tt[m];
    for (int i = 0; i < g->n; i++)
        tt[NIN + i] = eval_lut(tt[g->in[i][0]], tt[g->in[i][1]], tt[g->in[i][2]], g->imm[i]);
}

static int correct(const geno_t* g, const tt_t* tt) {
    for (int t = 0; t < 4; t++) {
        tt_t v = tt[g->out[t] >> 1];
        if (g->out[t] & 1) v = ~v;
        if (v != g_target[t]) return 0;
    }
    return 1;
}

static int active_count(const geno_t* g, uint8_t* act) {
    memset(act, 0, NIN + MAXG);
    for (int t = 0; t < 4; t++) act[g->out[t] >> 1] = 1;
    int cnt = 0;
    for (int i = g->n - 1; i >= 0; i--) {
        if (!act[NIN + i]) continue;
        cnt++;
        for (int q = 0; q < 3; q++) act[g->in[i][q]] = 1;
    }
    return cnt;
}

static void setup_targets(int sbox) {
    for (int m = 0; m < NIN; m++) {
        g_in_tt[m] = 0;
        for (int p = 0; p < 64; p++)
            if ((p >> (5 - m)) & 1) g_in_tt[m] |= (tt_t)1 << p;
    }
    for (int t = 0; t < 4; t++) {
        g_target[t] = 0;
        for (int x = 0; x < 64; x++) {
            int s = SBOX[sbox - 1][((x >> 5) & 1) * 2 + (x & 1)][(x >> 1) & 15];
            if ((s >> (3 - t)) & 1) g_target[t] |= (tt_t)1 << x;
        }
    }
}

/* ---- minimal reader for sboxgen's JSON: {"sbox": k, "gates": [[a,b,c,imm],...], "outputs": [..]} ---- */
static int next_int(const char** p, const char* end) {
    while (*p < end && !(**p >= '0' && **p <= '9')) (*p)++;
    int v = 0;
    while (*p < end && **p >= '0' && **p <= '9') v = v * 10 + (*(*p)++ - '0');
    return v;
}

static int read_circuit(const char* path, int sbox, geno_t* g) {
    FILE* f = fopen(path, "rb");
    if (!f) return 0;
    static char buf[1 << 20];
    size_t len = fread(buf, 1, sizeof(buf) - 1, f);
    fclose(f);
    buf[len] = 0;
    const char* p = buf;
    while ((p = strstr(p, "\"sbox\"")) != NULL) {
        const char* q = p + 6;
        int k = next_int(&q, buf + len);
        const char* gs = strstr(q, "\"gates\"");
        const char* os = strstr(q, "\"outputs\"");
        const char* nx = strstr(q, "\"sbox\"");
        if (!gs || !os) return 0;
        if (k == sbox) {
            const char* ge = os;
            g->n = 0;
            const char* r = gs + 7;
            for (;;) {
                const char* t = r;
                while (t < ge && !(*t >= '0' && *t <= '9')) t++;
                if (t >= ge) break;
                if (g->n >= MAXG) return 0;
                for (int q2 = 0; q2 < 3; q2++) g->in[g->n][q2] = (uint8_t)next_int(&r, ge);
                g->imm[g->n] = (uint8_t)next_int(&r, ge);
                g->n++;
            }
            const char* oe = nx ? nx : buf + len;
            r = os + 9;
            for (int t = 0; t < 4; t++) g->out[t] = next_int(&r, oe);
            return 1;
        }
        p = nx ? nx : buf + len;
        if (!nx) break;
    }
    return 0;
}

/* drop inactive gates, keep order; returns the compacted genome */
static geno_t compact(const geno_t* g) {
    uint8_t act[NIN + MAXG];
    active_count(g, act);
    int map[NIN + MAXG];
    for (int m = 0; m < NIN; m++) map[m] = m;
    geno_t c;
    c.n = 0;
    for (int i = 0; i < g->n; i++) {
        if (!act[NIN + i]) continue;
        map[NIN + i] = NIN + c.n;
        for (int q = 0; q < 3; q++) c.in[c.n][q] = (uint8_t)map[g->in[i][q]];
        c.imm[c.n] = g->imm[i];
        c.n++;
    }
    for (int t = 0; t < 4; t++) c.out[t] = 2 * map[g->out[t] >> 1] + (g->out[t] & 1);
    return c;
}

/* independent re-check against the table, point by point */
static int verify_table(const geno_t* g, int sbox) {
    for (int x = 0; x < 64; x++) {
        int val[NIN + MAXG];
        for (int m = 0; m < NIN; m++) val[m] = (x >> (5 - m)) & 1;
        for (int i = 0; i < g->n; i++)
            val[NIN + i] = (g->imm[i] >> (4 * val[g->in[i][0]] + 2 * val[g->in[i][1]] + val[g->in[i][2]])) & 1;
        int s = SBOX[sbox - 1][((x >> 5) & 1) * 2 + (x & 1)][(x >> 1) & 15];
        for (int t = 0; t < 4; t++)
            if ((val[g->out[t] >> 1] ^ (g->out[t] & 1)) != ((s >> (3 - t)) & 1)) return 0;
    }
    return 1;
}

static void write_circuit(const char* path, const geno_t* g, int sbox) {
    char tmp[4096];
    snprintf(tmp, sizeof tmp, "%s.tmp", path);
    FILE* f = fopen(tmp, "w");
    if (!f) return;
    fprintf(f, "[\n {\"sbox\": %d, \"gates\": [", sbox);
    for (int i = 0; i < g->n; i++)
        fprintf(f, "%s[%d, %d, %d, %d]", i ? ", " : "", g->in[i][0], g->in[i][1], g->in[i][2], g->imm[i]);
    fprintf(f, "], \"outputs\": [%d, %d, %d, %d]}\n]\n", g->out[0], g->out[1], g->out[2], g->out[3]);
    fclose(f);
    rename(tmp, path);
}

/* a spare gate with random inputs and function, inserted at a random
 * position (later gates and the outputs are renumbered) */
static void add_spare(geno_t* g) {
    int pos = rndn(g->n + 1);
    for (int i = g->n; i > pos; i--) {
        for (int q = 0; q < 3; q++) g->in[i][q] = g->in[i - 1][q];
        g->imm[i] = g->imm[i - 1];
    }
    g->n++;
    for (int i = pos + 1; i < g->n; i++)
        for (int q = 0; q < 3; q++)
            if (g->in[i][q] >= NIN + pos) g->in[i][q]++;
    for (int t = 0; t < 4; t++)
        if ((g->out[t] >> 1) >= NIN + pos) g->out[t] += 2;
    for (int q = 0; q < 3; q++) g->in[pos][q] = (uint8_t)rndn(NIN + pos);
    g->imm[pos] = (uint8_t)rnd();
}

static void mutate(geno_t* g, const tt_t* tt) {
    int genes = 4 * g->n + 4;
    int k = 1 + rndn(3);
    for (int h = 0; h < k; h++) {
        int x = rndn(genes);
        if (x >= 4 * g->n) {  /* output reference */
            g->out[x - 4 * g->n] = 2 * rndn(NIN + g->n) + (int)(rnd() & 1);
            continue;
        }
        int i = x >> 2, q = x & 3;
        if (q == 3) {
            g->imm[i] ^= (uint8_t)(1u << rndn(8));
            continue;
        }
        int old = g->in[i][q];
        int nw = rndn(NIN + i);
        g->in[i][q] = (uint8_t)nw;
        if (rnd() & 1) {  /* neutral rewiring when the new inputs allow it */
            int imm = lut_fit(tt[g->in[i][0]], tt[g->in[i][1]], tt[g->in[i][2]], tt[NIN + i]);
            if (imm >= 0) g->imm[i] = (uint8_t)imm;
            else g->in[i][q] = (uint8_t)old;
        }
    }
}

int main(int argc, char** argv) {
    if (argc < 7) {
        fprintf(stderr, "usage: %s in.json sbox seed seconds spare out.json [slack [drift.json]]\n", argv[0]);
        return 2;
    }
    int sbox = atoi(argv[2]);
    g_rng ^= (uint64_t)strtoull(argv[3], NULL, 10) * 0x2545F4914F6CDD1Dull;
    double seconds = atof(argv[4]);
    int spare = atoi(argv[5]);
    int slack = argc > 7 ? atoi(argv[7]) : 0;
    const char* outp = argv[6];
    if (sbox < 1 || sbox > 8) return 2;
    setup_targets(sbox);
    geno_t best;
    if (!read_circuit(argv[1], sbox, &best)) {
        fprintf(stderr, "no circuit for S%d in %s\n", sbox, argv[1]);
        return 1;
    }
    tt_t tt[NIN + MAXG];
    uint8_t act[NIN + MAXG];
    eval_all(&best, tt);
    if (!correct(&best, tt) || !verify_table(&best, sbox)) {
        fprintf(stderr, "start circuit for S%d is wrong\n", sbox);
        return 1;
    }
    best = compact(&best);
    int best_n = best.n;
    fprintf(stderr, "S%d: start %d gates\n", sbox, best_n);

    geno_t parent = best;
    while (parent.n < best_n + spare && parent.n < MAXG) add_spare(&parent);
    eval_all(&parent, tt);
    int parent_cost = active_count(&parent, act);
    clock_t t0 = clock();
    uint64_t gen = 0;
    const int lambda = 4;
    while ((double)(clock() - t0) / CLOCKS_PER_SEC < seconds) {
        geno_t bestc;
        int bestc_cost = 1 << 30;
        for (int l = 0; l < lambda; l++) {
            geno_t c = parent;
            mutate(&c, tt);
            tt_t ct[NIN + MAXG];
            eval_all(&c, ct);
            if (!correct(&c, ct)) continue;
            int cost = active_count(&c, act);
            if (cost <= bestc_cost) {
                bestc = c;
                bestc_cost = cost;
            }
        }
        /* with slack > 0, a slightly larger circuit is accepted now and
         * then (one offspring in ~4000), never more than slack gates above
         * the best, so the search can leave a local minimum */
        int up = slack > 0 && bestc_cost <= best_n + slack && (rnd() & 4095) == 0;
        if (bestc_cost <= parent_cost || (bestc_cost < (1 << 30) && up)) {
            parent = bestc;
            parent_cost = bestc_cost;
            eval_all(&parent, tt);
            if (parent_cost < best_n) {
                geno_t c = compact(&parent);
                if (verify_table(&c, sbox)) {
                    best = c;
                    best_n = c.n;
                    write_circuit(outp, &best, sbox);
                    fprintf(stderr, "S%d: %d gates (generation %llu)\n", sbox, best_n, (unsigned long long)gen);
                    /* refill spare gates for further drift */
                    parent = best;
                    while (parent.n < best_n + spare && parent.n < MAXG) add_spare(&parent);
                    eval_all(&parent, tt);
                    parent_cost = active_count(&parent, act);
                }
            }
        }
        gen++;
    }
    if (argc > 8) {  /* the circuit the search drifted to, as a start point for other searches */
        geno_t c = compact(&parent);
        if (verify_table(&c, sbox)) write_circuit(argv[8], &c, sbox);
    }
    fprintf(stderr, "S%d: done, %d gates after %llu generations\n", sbox, best_n, (unsigned long long)gen);
    return 0;
}
