/*
 * resub3.c -- exhaustive three-gate resubstitution for LOP3 S-box circuits.
 *
 * For every gate r whose maximum fanout-free cone (the gates that die with
 * it) holds four or more gates, look for
 *
 *     r = L3(L1(a, b, c), L2(d, e, f), x)
 *
 * with a..f and x any nodes outside that cone that do not depend on r, and
 * L1, L2, L3 any 3-input functions.  A hit replaces the cone by three gates.
 * The search is exhaustive over x and the two triples: the 64 input points
 * fall into cells (x, abc, def); r must be constant on every cell, and then
 * L1 and L2 must exist, which is a small two-colouring problem per choice of
 * L1.  Outputs may come out complemented (the consumer absorbs it).
 *
 *   gcc -O2 -o resub3 resub3.c
 *   ./resub3 in.json sbox out.json
 * The result is re-verified on all 64 inputs against the S-box table and
 * written only when it has fewer gates.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

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

typedef struct {
    int n;  /* nodes 0..5 are the inputs */
    int in[MAXN][3];
    int imm[MAXN];
    tt_t tt[MAXN];
    int out[4];
} circ_t;

static tt_t eval_lut(tt_t a, tt_t b, tt_t c, int imm) {
    tt_t r = 0;
    for (int k = 0; k < 8; k++)
        if ((imm >> k) & 1) r |= ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c);
    return r;
}

static void eval_all(circ_t* c) {
    for (int m = 0; m < 6; m++) {
        c->tt[m] = 0;
        for (int p = 0; p < 64; p++)
            if ((p >> (5 - m)) & 1) c->tt[m] |= (tt_t)1 << p;
    }
    for (int n = 6; n < c->n; n++) c->tt[n] = eval_lut(c->tt[c->in[n][0]], c->tt[c->in[n][1]], c->tt[c->in[n][2]], c->imm[n]);
}

static int verify(const circ_t* c, int box) {
    for (int p = 0; p < 64; p++) {
        int val[MAXN];
        for (int m = 0; m < 6; m++) val[m] = (p >> (5 - m)) & 1;
        for (int n = 6; n < c->n; n++)
            val[n] = (c->imm[n] >> (4 * val[c->in[n][0]] + 2 * val[c->in[n][1]] + val[c->in[n][2]])) & 1;
        const int s = SBOX[box][((p >> 5) & 1) * 2 + (p & 1)][(p >> 1) & 15];
        for (int t = 0; t < 4; t++)
            if ((val[c->out[t] >> 1] ^ (c->out[t] & 1)) != ((s >> (3 - t)) & 1)) return 0;
    }
    return 1;
}

static int read_num(const char** p, const char* end) {
    while (*p < end && !(**p >= '0' && **p <= '9')) (*p)++;
    int v = 0;
    while (*p < end && **p >= '0' && **p <= '9') v = v * 10 + (*(*p)++ - '0');
    return v;
}

static int load(const char* path, int box, circ_t* c) {
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
            c->n = 6;
            const char* r = gs + 7;
            for (;;) {
                const char* t = r;
                while (t < os && !(*t >= '0' && *t <= '9')) t++;
                if (t >= os || c->n >= MAXN) break;
                for (int z = 0; z < 3; z++) c->in[c->n][z] = read_num(&r, os);
                c->imm[c->n] = read_num(&r, os);
                c->n++;
            }
            r = os + 9;
            for (int t = 0; t < 4; t++) c->out[t] = read_num(&r, nx ? nx : buf + len);
            eval_all(c);
            return verify(c, box);
        }
        p = nx ? nx : buf + len;
        if (!nx) break;
    }
    return 0;
}

/* Marks r's maximum fanout-free cone; returns its size. */
static int mffc(const circ_t* c, int r, char* cone) {
    memset(cone, 0, MAXN);
    cone[r] = 1;
    int size = 1, changed = 1;
    while (changed) {
        changed = 0;
        for (int n = r - 1; n >= 6; n--) {
            if (cone[n]) continue;
            int is_out = 0;
            for (int t = 0; t < 4; t++) if ((c->out[t] >> 1) == n) is_out = 1;
            if (is_out) continue;
            int uses = 0, inside = 1;
            for (int h = n + 1; h < c->n; h++)
                for (int z = 0; z < 3; z++)
                    if (c->in[h][z] == n) { uses++; if (!cone[h]) inside = 0; }
            if (uses && inside) { cone[n] = 1; size++; changed = 1; }
        }
    }
    return size;
}

/* Given per-cell values of r (cell = x * 64 + u * 8 + v; -1 empty), find
 * L1 over u and L2 over v with r(cell) = L3(L1(u), L2(v), x).  Fills l1, l2
 * (8-bit truth tables over u and v) on success.
 *
 * For a choice of L1 the cells fall into four groups (x, L1(u)); in each
 * group r must depend on v alone.  A group where r takes both values needs
 * L2 to be r or its complement there, so every two of its v's must get L2
 * values differing exactly where their r values differ: parity constraints
 * between the eight v's, solved with a parity union-find. */
static int pfind(const int* par, const int* parity, int v, int* acc) {
    int p = 0;
    while (par[v] != v) { p ^= parity[v]; v = par[v]; }
    *acc = p;
    return v;
}

static int decompose(const int* cellv, int* l1, int* l2) {
    for (int g1 = 0; g1 < 128; g1++) { /* L3 absorbs a complement of L1 */
        int gval[4][8], ok = 1;
        memset(gval, 0xff, sizeof(gval));
        for (int x = 0; x < 2 && ok; x++)
            for (int u = 0; u < 8 && ok; u++)
                for (int v = 0; v < 8 && ok; v++) {
                    const int val = cellv[x * 64 + u * 8 + v];
                    if (val < 0) continue;
                    const int g = x * 2 + ((g1 >> u) & 1);
                    if (gval[g][v] < 0) gval[g][v] = val;
                    else if (gval[g][v] != val) ok = 0;
                }
        if (!ok) continue;
        int par[8], parity[8];
        for (int v = 0; v < 8; v++) { par[v] = v; parity[v] = 0; }
        for (int g = 0; g < 4 && ok; g++) {
            int has0 = 0, has1 = 0, v0 = -1;
            for (int v = 0; v < 8; v++) {
                if (gval[g][v] == 0) has0 = 1;
                if (gval[g][v] == 1) has1 = 1;
                if (gval[g][v] >= 0 && v0 < 0) v0 = v;
            }
            if (!(has0 && has1)) continue;
            for (int v = v0 + 1; v < 8 && ok; v++) {
                if (gval[g][v] < 0) continue;
                const int want = gval[g][v0] ^ gval[g][v];
                int pa, pb;
                const int ra = pfind(par, parity, v0, &pa), rb = pfind(par, parity, v, &pb);
                if (ra == rb) {
                    if ((pa ^ pb) != want) ok = 0;
                } else {
                    par[rb] = ra;
                    parity[rb] = pa ^ pb ^ want;
                }
            }
        }
        if (!ok) continue;
        int g2 = 0;
        for (int v = 0; v < 8; v++) {
            int pv;
            pfind(par, parity, v, &pv);
            if (pv) g2 |= 1 << v;
        }
        *l1 = g1;
        *l2 = g2;
        return 1;
    }
    return 0;
}

static int try_node(circ_t* c, int r, int box) {
    char cone[MAXN], tfo[MAXN] = {0};
    const int m = mffc(c, r, cone);
    if (m < 4) return 0;
    for (int n = r + 1; n < c->n; n++)
        for (int z = 0; z < 3; z++)
            if (c->in[n][z] == r || tfo[c->in[n][z]]) tfo[n] = 1;
    int av[MAXN], na = 0;
    for (int n = 0; n < c->n; n++)
        if (!cone[n] && !tfo[n]) av[na++] = n;
    const tt_t target = c->tt[r];
    /* every ordered choice: x, then triples T1 < T2 */
    int ntri = 0;
    static int tri[MAXN * MAXN * MAXN / 6 + 8][3];
    for (int i = 0; i < na; i++)
        for (int j = i + 1; j < na; j++)
            for (int k = j + 1; k < na; k++) { tri[ntri][0] = av[i]; tri[ntri][1] = av[j]; tri[ntri][2] = av[k]; ntri++; }
    for (int xi = 0; xi < na; xi++) {
        const tt_t tx = c->tt[av[xi]];
        for (int t1 = 0; t1 < ntri; t1++) {
            tt_t cls[16]; /* (x, u) classes */
            const tt_t a = c->tt[tri[t1][0]], b = c->tt[tri[t1][1]], cc = c->tt[tri[t1][2]];
            for (int u = 0; u < 8; u++) {
                const tt_t mu = ((u & 4) ? a : ~a) & ((u & 2) ? b : ~b) & ((u & 1) ? cc : ~cc);
                cls[u] = mu & ~tx;
                cls[8 + u] = mu & tx;
            }
            for (int t2 = t1 + 1; t2 < ntri; t2++) {
                const tt_t td = c->tt[tri[t2][0]], te = c->tt[tri[t2][1]], tf = c->tt[tri[t2][2]];
                tt_t mv[8];
                for (int v = 0; v < 8; v++) mv[v] = ((v & 4) ? td : ~td) & ((v & 2) ? te : ~te) & ((v & 1) ? tf : ~tf);
                int bad = 0, cellv[128];
                for (int xu = 0; xu < 16 && !bad; xu++) {
                    const tt_t cu = cls[xu];
                    for (int v = 0; v < 8; v++) {
                        const tt_t cell = cu & mv[v];
                        int val = -1;
                        if (cell) {
                            if ((cell & target) && (cell & ~target)) { bad = 1; break; }
                            val = (cell & target) ? 1 : 0;
                        }
                        cellv[(xu >> 3) * 64 + (xu & 7) * 8 + v] = val;
                    }
                }
                if (bad) continue;
                int l1, l2;
                if (!decompose(cellv, &l1, &l2)) continue;
                /* build: the nodes outside the cone that do not depend on
                 * r, then g1 = L1(T1), g2 = L2(T2), r' = L3(g1, g2, x),
                 * then the nodes that read r (a topological order) */
                circ_t t;
                int map[MAXN];
                t.n = 6;
                for (int q = 0; q < 6; q++) map[q] = q;
                for (int n = 6; n < c->n; n++) {
                    map[n] = -1;
                    if (cone[n] || tfo[n]) continue;
                    const int k = t.n++;
                    for (int z = 0; z < 3; z++) t.in[k][z] = map[c->in[n][z]];
                    t.imm[k] = c->imm[n];
                    map[n] = k;
                }
                const int g1 = t.n++, g2 = t.n++, g3 = t.n++;
                for (int z = 0; z < 3; z++) { t.in[g1][z] = map[tri[t1][z]]; t.in[g2][z] = map[tri[t2][z]]; }
                t.imm[g1] = l1;
                t.imm[g2] = l2;
                t.in[g3][0] = g1; t.in[g3][1] = g2; t.in[g3][2] = map[av[xi]];
                t.imm[g3] = 0;
                map[r] = g3;
                for (int n = r + 1; n < c->n; n++) {
                    if (!tfo[n]) continue;
                    const int k = t.n++;
                    for (int z = 0; z < 3; z++) t.in[k][z] = map[c->in[n][z]];
                    t.imm[k] = c->imm[n];
                    map[n] = k;
                }
                int order_ok = 1;
                for (int n = 6; n < t.n; n++)
                    for (int z = 0; z < 3; z++)
                        if (t.in[n][z] < 0 || t.in[n][z] >= n) order_ok = 0;
                if (!order_ok) continue;
                eval_all(&t);
                const tt_t g1t = t.tt[g1], g2t = t.tt[g2], xt = t.tt[t.in[g3][2]];
                int imm3 = 0, okfit = 1;
                for (int k = 0; k < 8 && okfit; k++) {
                    const tt_t sel = ((k & 4) ? g1t : ~g1t) & ((k & 2) ? g2t : ~g2t) & ((k & 1) ? xt : ~xt);
                    if (sel & target) { if (sel & ~target) okfit = 0; else imm3 |= 1 << k; }
                }
                if (!okfit) continue;
                t.imm[g3] = imm3;
                for (int tt_ = 0; tt_ < 4; tt_++) t.out[tt_] = 2 * map[c->out[tt_] >> 1] + (c->out[tt_] & 1);
                eval_all(&t);
                if (!verify(&t, box)) continue;
                /* drop gates that no longer feed an output */
                int live[MAXN] = {0};
                for (int q = 0; q < 4; q++) live[t.out[q] >> 1] = 1;
                for (int n = t.n - 1; n >= 6; n--) if (live[n]) for (int z = 0; z < 3; z++) live[t.in[n][z]] = 1;
                circ_t d;
                int mp[MAXN];
                d.n = 6;
                for (int q = 0; q < 6; q++) mp[q] = q;
                for (int n = 6; n < t.n; n++) {
                    if (!live[n]) continue;
                    const int k = d.n++;
                    for (int z = 0; z < 3; z++) d.in[k][z] = mp[t.in[n][z]];
                    d.imm[k] = t.imm[n];
                    mp[n] = k;
                }
                for (int q = 0; q < 4; q++) d.out[q] = 2 * mp[t.out[q] >> 1] + (t.out[q] & 1);
                eval_all(&d);
                if (d.n < c->n && verify(&d, box)) {
                    fprintf(stderr, "S%d: node %d (cone %d) -> 3 gates: %d -> %d gates\n", box + 1, r, m, c->n - 6,
                            d.n - 6);
                    *c = d;
                    return 1;
                }
            }
        }
    }
    return 0;
}

int main(int argc, char** argv) {
    if (argc < 4) {
        fprintf(stderr, "usage: %s in.json sbox out.json\n", argv[0]);
        return 2;
    }
    const int box = atoi(argv[2]) - 1;
    if (box < 0 || box > 7) return 2;
    static circ_t c;
    if (!load(argv[1], box, &c)) {
        fprintf(stderr, "no valid circuit for S%d\n", box + 1);
        return 1;
    }
    const int start = c.n - 6;
    fprintf(stderr, "S%d: start %d gates\n", box + 1, start);
    int improved = 1;
    while (improved) {
        improved = 0;
        for (int r = c.n - 1; r >= 6 && !improved; r--) improved = try_node(&c, r, box);
    }
    if (c.n - 6 < start) {
        FILE* f = fopen(argv[3], "w");
        if (!f) return 1;
        fprintf(f, "[{\"sbox\": %d, \"gates\": [", box + 1);
        for (int n = 6; n < c.n; n++)
            fprintf(f, "%s[%d, %d, %d, %d]", n > 6 ? ", " : "", c.in[n][0], c.in[n][1], c.in[n][2], c.imm[n]);
        fprintf(f, "], \"outputs\": [%d, %d, %d, %d]}]\n", c.out[0], c.out[1], c.out[2], c.out[3]);
        fclose(f);
    }
    fprintf(stderr, "S%d: done, %d gates\n", box + 1, c.n - 6);
    return 0;
}
