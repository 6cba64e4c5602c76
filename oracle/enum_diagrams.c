/*
 * Brute-force enumeration of self-energy diagram topologies (oracle; test
 * infrastructure only, never linked into the product library).
 *
 * Follows the paper's Sec. II.A (Eq. sigma_integration): an order-n term has n
 * instantaneous interaction lines (2n vertices) and the sum runs over all
 * distinct topologies.  Here a Green's-function contraction is a permutation
 * sigma of {0..2n-1, X}: vertex v sends its outgoing fermion line to sigma(v),
 * the external point X feeds the in-vertex sigma(X) and receives the line from
 * the out-vertex.  Interaction line i joins vertices 2i and 2i+1.
 *
 * Every permutation with sigma(X) = 0 is visited (the relabelling symmetry of
 * interaction lines and of their two ends is transitive on vertices, so every
 * topology is met), reduced to a canonical form by a deterministic traversal,
 * and counted in a hash set.  For each distinct connected topology the program
 * prints:  multiplicity F is1PI tadpole_free sigma'(0) ... sigma'(2n-1)
 * where sigma' is the canonical permutation (X printed as 2n), F the number of
 * closed fermion loops.  Multiplicity must be (n-1)! 2^(n-1) for every topology
 * (no automorphisms once the external legs are fixed) -- the tests check it.
 *
 * Canonical traversal: start at X, follow fermion lines; the first time a
 * vertex of an unlabelled interaction line is met, that line gets the next
 * label L, the met vertex becomes 2L and its partner 2L+1.  After the open path
 * returns to X, the unvisited vertex with the smallest canonical label starts
 * the next closed loop, and so on.  A contraction whose traversal leaves a line
 * unlabelled is disconnected and is skipped.
 *
 * Usage: enum_diagrams n   (1 <= n <= 6)
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXV 14

static int n_ord, nv, XN;

typedef struct {
    uint64_t key;
    uint64_t count;
} slot_t;

static slot_t *table;
static uint64_t table_mask;
static uint64_t n_unique;

static uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void table_add(uint64_t key) {
    uint64_t h = mix64(key) & table_mask;
    for (;;) {
        if (table[h].count == 0) {
            table[h].key = key;
            table[h].count = 1;
            n_unique++;
            if (n_unique * 2 > table_mask) {
                fprintf(stderr, "hash table too small\n");
                exit(2);
            }
            return;
        }
        if (table[h].key == key) {
            table[h].count++;
            return;
        }
        h = (h + 1) & table_mask;
    }
}

/* sigma[v] for v in 0..nv-1 gives the target (XN for the external point). */
static int canonical(const int *sigma, int *out_sigma) {
    int cid[MAXV], visited[MAXV], nl = 0;
    for (int v = 0; v < nv; v++) { cid[v] = -1; visited[v] = 0; }
    int v = 0; /* sigma(X) = 0 */
    while (v != XN) {
        if (cid[v] < 0) { cid[v] = 2 * nl; cid[v ^ 1] = 2 * nl + 1; nl++; }
        visited[v] = 1;
        v = sigma[v];
    }
    for (;;) {
        int best = -1, bestid = 1 << 30;
        for (int u = 0; u < nv; u++)
            if (!visited[u] && cid[u] >= 0 && cid[u] < bestid) { best = u; bestid = cid[u]; }
        if (best < 0) break;
        int u = best;
        do {
            if (cid[u] < 0) { cid[u] = 2 * nl; cid[u ^ 1] = 2 * nl + 1; nl++; }
            visited[u] = 1;
            u = sigma[u];
        } while (u != best);
    }
    if (nl < n_ord) return 0;
    for (int u = 0; u < nv; u++) out_sigma[cid[u]] = (sigma[u] == XN) ? XN : cid[sigma[u]];
    return 1;
}

static uint64_t pack(const int *s) {
    uint64_t k = 0;
    for (int v = 0; v < nv; v++) k |= ((uint64_t)s[v]) << (4 * v);
    return k;
}

static void unpack(uint64_t k, int *s) {
    for (int v = 0; v < nv; v++) s[v] = (int)((k >> (4 * v)) & 15u);
}

/* union-find over vertices */
static int uf[MAXV];
static int uf_find(int a) { while (uf[a] != a) a = uf[a] = uf[uf[a]]; return a; }
static void uf_union(int a, int b) { a = uf_find(a); b = uf_find(b); if (a != b) uf[a] = b; }

/* connected after removing fermion edge (skip_g = source vertex) or
 * interaction line (skip_v = line index); returns 1 if a single component */
static int connected_without(const int *s, int skip_g, int skip_v) {
    for (int v = 0; v < nv; v++) uf[v] = v;
    for (int v = 0; v < nv; v++)
        if (s[v] != XN && v != skip_g) uf_union(v, s[v]);
    for (int i = 0; i < n_ord; i++)
        if (i != skip_v) uf_union(2 * i, 2 * i + 1);
    int r = uf_find(0);
    for (int v = 1; v < nv; v++) if (uf_find(v) != r) return 0;
    return 1;
}

int main(int argc, char **argv) {
    if (argc < 2) { fprintf(stderr, "usage: %s n\n", argv[0]); return 1; }
    n_ord = atoi(argv[1]);
    if (n_ord < 1 || n_ord > 6) { fprintf(stderr, "n out of range\n"); return 1; }
    nv = 2 * n_ord;
    XN = nv;
    uint64_t tsize = 1ull << 22;
    table = (slot_t *)calloc(tsize, sizeof(slot_t));
    table_mask = tsize - 1;

    /* targets for sources 0..nv-1: {1..nv-1, X}; iterate all orderings
     * with Heap's algorithm */
    int tgt[MAXV], c[MAXV], cs[MAXV];
    for (int i = 0; i < nv - 1; i++) tgt[i] = i + 1;
    tgt[nv - 1] = XN;
    for (int i = 0; i < nv; i++) c[i] = 0;
    uint64_t n_perm = 0;
    if (canonical(tgt, cs)) table_add(pack(cs));
    n_perm++;
    int i = 1;
    while (i < nv) {
        if (c[i] < i) {
            int j = (i % 2 == 0) ? 0 : c[i];
            int t = tgt[j]; tgt[j] = tgt[i]; tgt[i] = t;
            if (canonical(tgt, cs)) table_add(pack(cs));
            n_perm++;
            c[i]++;
            i = 1;
        } else {
            c[i] = 0;
            i++;
        }
    }
    fprintf(stderr, "n=%d permutations=%llu unique_connected=%llu\n", n_ord,
            (unsigned long long)n_perm, (unsigned long long)n_unique);

    for (uint64_t h = 0; h <= table_mask; h++) {
        if (table[h].count == 0) continue;
        int s[MAXV];
        unpack(table[h].key, s);
        /* closed loops: cycles of s not through X */
        int seen[MAXV] = {0}, F = 0, v = 0;
        while (v != XN) { seen[v] = 1; v = s[v]; }
        for (int u = 0; u < nv; u++) {
            if (seen[u]) continue;
            F++;
            int w = u;
            do { seen[w] = 1; w = s[w]; } while (w != u);
        }
        /* 1PI: removing any fermion line of the open path keeps it connected */
        int onepi = 1;
        v = 0;
        while (s[v] != XN) {
            if (!connected_without(s, v, -1)) { onepi = 0; break; }
            v = s[v];
        }
        /* tadpole: an interaction line whose removal disconnects the diagram */
        int tadfree = 1;
        for (int l = 0; l < n_ord; l++)
            if (!connected_without(s, -1, l)) { tadfree = 0; break; }
        printf("%llu %d %d %d", (unsigned long long)table[h].count, F, onepi, tadfree);
        for (int u = 0; u < nv; u++) printf(" %d", s[u]);
        printf("\n");
    }
    free(table);
    return 0;
}
