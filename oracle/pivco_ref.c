/*
 * PivCo-Huffman CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the PivCo-Huffman method that the GPU library is checked
 * against.  Only the tests, the smoke check and the benchmark's CPU-baseline /
 * reference leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes, step by step (each function cites its passage):
 *   1. histogram of a block                        (Sec. 4, "symbol frequency counting")
 *   2. length-limited code lengths, L = 11         (Sec. 1.2; App. D) -- optimal
 *      package-merge; the paper names no algorithm, see the readings below
 *   3. canonical codes                             (Sec. 1 note on canonical coding; App. D)
 *   3b. optionally, the regrouped (non-canonical) tree with flat subtrees:
 *      equal-length symbols combined in power-of-two groups, each group of
 *      2^D >= 4 symbols one flat node             (Sec. 2.2.3, 2.2.4; App. D)
 *   4. the pivoted tree: one node per proper code prefix, bit 1 = right
 *                                                  (Listing 1; Sec. 2, Fig. 2-3)
 *   5. per-node bitmaps, LSB-first inside bytes; a flat node stores the
 *      D-bit index of each of its symbols, packed (Sec. 2; Sec. 2.4.2 bit_pos
 *      table; Sec. 2.2.3 scatter_flat_D; App. D flat subtree roots)
 *   6. selective ANS: node selection rule and byte-wise static-table ANS
 *                                                  (Sec. 5.2; App. D marker byte)
 *   7. the block record (wire format)              (App. D, adapted: see below)
 *   8. decode by the definition: a per-node cursor walk (Listing 1 applied to
 *      the pivoted layout, Sec. 2)
 *   9. PivCo-Golomb: the unary (Golomb parameter 1) code pivoted into a list
 *      of bitmaps, its record and its decode by the definition (App. G)
 *
 * Readings where the paper is silent or loose (each is part of the format):
 *   R1  code lengths: optimal package-merge; leaves ordered by (count, symbol),
 *       a leaf sorts before a package of equal weight, packages keep creation
 *       order; the first 2K-2 items of the shallowest list are selected.
 *   R2  canonical order: (length, symbol) ascending, consecutive integers,
 *       most significant bit first.
 *   R3  node order: breadth-first (depth, then prefix value ascending).
 *   R4  bitmap bit j lives in byte j>>3 at bit (j&7); pad bits are 0.
 *   R5  ANS: rANS over bitmap BYTES with 50 static tables t = 50..99 built for
 *       i.i.d. bits with P(bit = 0) = t/100; frequencies depend only on the
 *       byte's popcount class (exact integers, M = 2^15, byte 0x00 absorbs the
 *       rounding slack); 32-bit state in [2^16, 2^32), 16-bit renormalisation
 *       words; bitmaps split into 16 KiB segments, each with W = min(32,
 *       max(1, ceil(bytes/512))) interleaved states, byte j -> state j mod W.
 *   R6  ANS selection: ceil(n/8) >= 32 bytes, skew = max(n0,n1)/n > 0.625,
 *       (depth + fseH)/(depth + 1) < 0.95 with fseH in Q16; table
 *       t = round-half-up(100*skew) clamped to 50..99; XOR flag when n1 > n0;
 *       if the ANS body is not smaller than the raw bitmap, the raw bitmap is
 *       stored with marker 0xFF.
 *   R7  record: u32 widths, a node directory of u32 counts, ANS bodies after
 *       all raw bodies, records padded to 16 bytes.
 *   R8  PivCo-Golomb (App. G names Golomb coding and a list of bitmaps, and
 *       decodes a 1 bit to 0x00 and a 0 bit to the child's value plus 1):
 *       Golomb parameter 1, i.e. unary codes with stop bit 1; values are
 *       bytes; bitmap j holds the bit of every value >= j; a "PVG1" record
 *       with u32 counts n_j like R7.
 *   R10 flat subtrees (Sec. 2.2.3-2.2.4 describe the regrouping in words):
 *       code lengths are those of R1.  For each length l the symbols of that
 *       length, ascending, are cut greedily into groups of the largest power
 *       of two 2^D that is left (first 2^D symbols first); a group is one item
 *       of length l - D.  Items get canonical codes in (length, first symbol)
 *       order; symbol number x of a group (ascending) has the code
 *       (item code << D) | x, so every symbol keeps its length.  A group with
 *       D >= 2 is a flat node (a group of two is an ordinary node with two
 *       leaves).  A flat node's body is its symbols' D-bit indices x in block
 *       order, value j at bits [jD, jD + D), least significant bit first
 *       (App. D: ceil(n*D/8) bytes).  Flat nodes are never ANS coded; their
 *       marker byte is 0xF0 + D, so body sizes follow from the record's
 *       tables alone, and their bodies sit with the raw ones.  Nodes
 *       (ordinary and flat) are ordered breadth-first as in R3.  Records of
 *       this tree carry the tag "PVC2" in place of "PVC1".
 *
 * Parity status: every function above is pinned by the oracle tests (worked
 * examples of Sec. 1.1 and 2.2, brute-force optimality, Kraft, closed forms
 * of Sec. 5.1, round trips; for PivCo-Golomb a hand-derived record, the plain
 * unary stream, closed forms of the counts and App. G's bottom-up merge).  The exact bytes of an ANS stream are pinned
 * only by this definition and the round trip: "parity unpinned" beyond that.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define REF_OK 0
#define REF_ERR_ARG 1
#define REF_ERR_CAPACITY 2
#define REF_ERR_CORRUPT 3

#define REF_MAX_LEN_CAP 15
#define REF_ANS_SCALE 15
#define REF_ANS_M (1u << REF_ANS_SCALE)
#define REF_ANS_L (1u << 16)
#define REF_ANS_SEG 16384u
#define REF_MARK_RAW_SEL 0xFFu
#define REF_MARK_FLAT 0xF0u       /* flat node of depth D: marker 0xF0 + D (R10) */

typedef struct ref_params {
    int32_t max_len;        /* L (App. D: 11) */
    int32_t ans_enable;     /* selective ANS on/off (Sec. 5.2) */
    int32_t ans_min_bytes;  /* PIVCO_FSE_MIN_BITMAP_BYTES, 32 */
    int32_t ans_skew_num;   /* PIVCO_FSE_MIN_THRESHOLD = num/den = 5/8 */
    int32_t ans_skew_den;
    int32_t ans_ratio_pct;  /* PIVCO_FSE_MIN_RATIO, 95 (%) */
    int32_t flat;           /* regrouped tree with flat subtrees (R10) on/off */
} ref_params;

/* ------------------------------------------------------------------ */
/* little-endian helpers                                               */
/* ------------------------------------------------------------------ */
static void put32(uint8_t *p, uint32_t v) {
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
static uint32_t get32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static void put16(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static uint32_t get16(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static int popcount8(unsigned b) { int c = 0; while (b) { c += b & 1u; b >>= 1; } return c; }

/* ------------------------------------------------------------------ */
/* 1. Histogram (Sec. 4: end-to-end encode is dominated by counting)   */
/* ------------------------------------------------------------------ */
int ref_histogram(const uint8_t *x, uint64_t n, uint32_t *hist) {
    for (int s = 0; s < 256; s++) hist[s] = 0;
    for (uint64_t i = 0; i < n; i++) hist[x[i]]++;
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* 2. Length-limited code lengths by package-merge (App. D: L = 11;    */
/*    reading R1).  Lists are built from the deepest level (L) up to   */
/*    level 1; each list is the sorted leaves merged with the packages */
/*    made by pairing neighbours of the list one level deeper.         */
/* ------------------------------------------------------------------ */
typedef struct pm_item {
    uint64_t w;      /* weight */
    int kind;        /* 0 = leaf, 1 = package */
    int key;         /* leaf: sorted leaf index; package: creation index */
    int a, b;        /* package: indices of its two items in the deeper list */
} pm_item;

static int pm_less(const pm_item *x, const pm_item *y) {
    if (x->w != y->w) return x->w < y->w;
    if (x->kind != y->kind) return x->kind < y->kind;   /* leaf first */
    return x->key < y->key;
}

/* count how often each leaf occurs inside item `it` of list `lvl` */
static void pm_expand(pm_item **lists, int lvl, int idx, int *cnt) {
    const pm_item *it = &lists[lvl][idx];
    if (it->kind == 0) { cnt[it->key]++; return; }
    pm_expand(lists, lvl + 1, it->a, cnt);
    pm_expand(lists, lvl + 1, it->b, cnt);
}

int ref_code_lengths(const uint32_t *hist, int max_len, uint8_t *lens) {
    int K = 0, sym[256];
    uint64_t f[256];
    for (int s = 0; s < 256; s++) lens[s] = 0;
    if (max_len < 1 || max_len > REF_MAX_LEN_CAP) return REF_ERR_ARG;
    for (int s = 0; s < 256; s++) if (hist[s]) { sym[K] = s; f[K] = hist[s]; K++; }
    if (K <= 1) return REF_OK;                 /* empty / constant block: no code */
    if (K > (1 << max_len)) return REF_ERR_ARG;
    /* sort leaves by (count, symbol): insertion sort, K <= 256 */
    for (int i = 1; i < K; i++) {
        int s = sym[i]; uint64_t w = f[i]; int j = i - 1;
        while (j >= 0 && (f[j] > w || (f[j] == w && sym[j] > s))) { f[j + 1] = f[j]; sym[j + 1] = sym[j]; j--; }
        f[j + 1] = w; sym[j + 1] = s;
    }
    pm_item **lists = (pm_item **)calloc((size_t)max_len + 2, sizeof(pm_item *));
    int *len_of = (int *)calloc((size_t)max_len + 2, sizeof(int));
    if (!lists || !len_of) { free(lists); free(len_of); return REF_ERR_ARG; }
    /* level L: the leaves alone */
    lists[max_len] = (pm_item *)calloc((size_t)K, sizeof(pm_item));
    for (int i = 0; i < K; i++) { pm_item it = { f[i], 0, i, -1, -1 }; lists[max_len][i] = it; }
    len_of[max_len] = K;
    for (int lvl = max_len - 1; lvl >= 1; lvl--) {
        int np = len_of[lvl + 1] / 2;         /* an odd last item is dropped */
        int tot = K + np;
        pm_item *cur = (pm_item *)calloc((size_t)tot, sizeof(pm_item));
        for (int i = 0; i < K; i++) { pm_item it = { f[i], 0, i, -1, -1 }; cur[i] = it; }
        for (int j = 0; j < np; j++) {
            const pm_item *x = &lists[lvl + 1][2 * j], *y = &lists[lvl + 1][2 * j + 1];
            pm_item it = { x->w + y->w, 1, j, 2 * j, 2 * j + 1 };
            cur[K + j] = it;
        }
        /* plain insertion sort by (weight, leaf-first, key) */
        for (int i = 1; i < tot; i++) {
            pm_item v = cur[i]; int j = i - 1;
            while (j >= 0 && pm_less(&v, &cur[j])) { cur[j + 1] = cur[j]; j--; }
            cur[j + 1] = v;
        }
        lists[lvl] = cur; len_of[lvl] = tot;
    }
    int cnt[256];
    memset(cnt, 0, sizeof(cnt));
    int take = 2 * K - 2;
    if (take > len_of[1]) take = len_of[1];
    for (int i = 0; i < take; i++) pm_expand(lists, 1, i, cnt);
    for (int i = 0; i < K; i++) lens[sym[i]] = (uint8_t)cnt[i];
    for (int lvl = 1; lvl <= max_len; lvl++) free(lists[lvl]);
    free(lists); free(len_of);
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* 3. Canonical codes (reading R2).  code[s] holds lens[s] bits, MSB   */
/*    is the first (root) decision.                                    */
/* ------------------------------------------------------------------ */
int ref_canonical_codes(const uint8_t *lens, uint32_t *codes) {
    int order[256], K = 0;
    for (int s = 0; s < 256; s++) { codes[s] = 0; if (lens[s]) order[K++] = s; }
    for (int i = 1; i < K; i++) {   /* sort by (len, sym) */
        int s = order[i], j = i - 1;
        while (j >= 0 && (lens[order[j]] > lens[s] || (lens[order[j]] == lens[s] && order[j] > s))) { order[j + 1] = order[j]; j--; }
        order[j + 1] = s;
    }
    uint32_t c = 0;
    for (int i = 0; i < K; i++) {
        if (i > 0) c = (c + 1) << (lens[order[i]] - lens[order[i - 1]]);
        codes[order[i]] = c;
    }
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* 3b. Regrouped codes (Sec. 2.2.4; reading R10).  Each length class    */
/*     is cut into power-of-two groups, largest first; the groups get   */
/*     canonical codes as items of length l - D; a symbol's code is its */
/*     group's code followed by its D-bit index in the group.           */
/*     fd[s] = D when the symbol's group is a flat node (D >= 2), else 0 */
/* ------------------------------------------------------------------ */
int ref_flat_codes(const uint8_t *lens, uint32_t *codes, int32_t *fd) {
    int glen[256], gD[256], gfirst[256], gsym[256], ng = 0, ns = 0;
    for (int s = 0; s < 256; s++) { codes[s] = 0; fd[s] = 0; }
    for (int l = 1; l <= REF_MAX_LEN_CAP; l++) {
        int mem[256], m = 0;
        for (int s = 0; s < 256; s++) if (lens[s] == l) mem[m++] = s;
        int at = 0;
        while (at < m) {
            int D = 0;
            while ((1 << (D + 1)) <= m - at) D++;
            if (D > l) return REF_ERR_ARG;              /* more symbols than codes of length l */
            glen[ng] = l - D; gD[ng] = D; gfirst[ng] = ns;
            for (int k = 0; k < (1 << D); k++) gsym[ns++] = mem[at + k];
            at += 1 << D;
            ng++;
        }
    }
    /* canonical codes of the items, ordered by (item length, first symbol) */
    int order[256];
    for (int i = 0; i < ng; i++) order[i] = i;
    for (int i = 1; i < ng; i++) {
        int g = order[i], j = i - 1;
        while (j >= 0 && (glen[order[j]] > glen[g] ||
                          (glen[order[j]] == glen[g] && gsym[gfirst[order[j]]] > gsym[gfirst[g]]))) {
            order[j + 1] = order[j]; j--;
        }
        order[j + 1] = g;
    }
    uint32_t c = 0;
    for (int i = 0; i < ng; i++) {
        int g = order[i];
        if (i > 0) c = (c + 1) << (glen[g] - glen[order[i - 1]]);
        for (int x = 0; x < (1 << gD[g]); x++) {
            int sy = gsym[gfirst[g] + x];
            codes[sy] = (c << gD[g]) | (uint32_t)x;
            fd[sy] = gD[g] >= 2 ? gD[g] : 0;
        }
    }
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* 4. The pivoted tree (Listing 1: bit 1 = right; Sec. 2: one bitmap   */
/*    per internal node = per proper code prefix).  Node order R3.     */
/*    With flat subtrees (R10) the prefixes at and below a flat group's */
/*    item code are replaced by one flat node of depth D whose symbol   */
/*    number x is the symbol coded (prefix << D) | x.                   */
/* ------------------------------------------------------------------ */
typedef struct ref_tree {
    int n_int;                 /* nodes: ordinary and flat */
    int depth[256];
    uint32_t prefix[256];
    int flat[256];             /* D of a flat node, 0 for an ordinary node */
    int child[256][2];         /* ordinary: >= 0 node id, < 0 leaf -(symbol+1) */
    uint8_t ftab[256][256];    /* flat: symbol of index x */
} ref_tree;

static int tree_find(const ref_tree *t, int d, uint32_t p) {
    for (int v = 0; v < t->n_int; v++) if (t->depth[v] == d && t->prefix[v] == p) return v;
    return -1;
}

/* the node a symbol's code bit d is read at (d below the flat depth), or
   its flat node (d = lens - fd) */
static int sym_node(const ref_tree *t, const uint8_t *lens, const uint32_t *codes, int s, int d) {
    return tree_find(t, d, codes[s] >> (lens[s] - d));
}

static int build_tree(const uint8_t *lens, const uint32_t *codes, const int32_t *fd, ref_tree *t) {
    /* collect the nodes (d, p, D): ordinary nodes are proper prefixes above
       a symbol's flat node, flat nodes are the flat groups' item codes */
    int nd = 0;
    int dd[4096], DD[4096]; uint32_t pp[4096];
    for (int s = 0; s < 256; s++) {
        if (!lens[s]) continue;
        int top = lens[s] - fd[s];
        for (int d = 0; d <= top; d++) {
            int D = d < top ? 0 : fd[s];
            if (d == top && fd[s] == 0) break;       /* a leaf, not a node */
            uint32_t p = codes[s] >> (lens[s] - d);
            int seen = -1;
            for (int k = 0; k < nd; k++) if (dd[k] == d && pp[k] == p) { seen = k; break; }
            if (seen >= 0) { if (DD[seen] != D) return REF_ERR_CORRUPT; continue; }
            if (nd >= 4096) return REF_ERR_ARG;
            dd[nd] = d; pp[nd] = p; DD[nd] = D; nd++;
        }
    }
    if (nd > 255) return REF_ERR_ARG;
    /* breadth-first order: sort by (depth, prefix) */
    for (int i = 1; i < nd; i++) {
        int d = dd[i], D = DD[i]; uint32_t p = pp[i]; int j = i - 1;
        while (j >= 0 && (dd[j] > d || (dd[j] == d && pp[j] > p))) { dd[j + 1] = dd[j]; pp[j + 1] = pp[j]; DD[j + 1] = DD[j]; j--; }
        dd[j + 1] = d; pp[j + 1] = p; DD[j + 1] = D;
    }
    t->n_int = nd;
    for (int v = 0; v < nd; v++) { t->depth[v] = dd[v]; t->prefix[v] = pp[v]; t->flat[v] = DD[v]; }
    for (int v = 0; v < nd; v++) {
        if (t->flat[v]) {
            /* symbol x of the flat node: code (prefix << D) | x, length depth + D */
            int D = t->flat[v];
            t->child[v][0] = t->child[v][1] = 0;
            for (int x = 0; x < (1 << D); x++) {
                int sym = -1;
                for (int s = 0; s < 256; s++)
                    if (lens[s] == t->depth[v] + D && fd[s] == D && codes[s] == ((t->prefix[v] << D) | (uint32_t)x)) { sym = s; break; }
                if (sym < 0) return REF_ERR_CORRUPT;
                t->ftab[v][x] = (uint8_t)sym;
            }
            continue;
        }
        for (int b = 0; b < 2; b++) {
            int cd = t->depth[v] + 1; uint32_t cp = (t->prefix[v] << 1) | (uint32_t)b;
            int id = tree_find(t, cd, cp);
            if (id >= 0) { t->child[v][b] = id; continue; }
            int leaf = -1;
            for (int s = 0; s < 256; s++) if (lens[s] == cd && fd[s] == 0 && codes[s] == cp) { leaf = s; break; }
            if (leaf < 0) return REF_ERR_CORRUPT;   /* not a full tree */
            t->child[v][b] = -leaf - 1;
        }
    }
    return REF_OK;
}

/* codes and tree of a block: canonical (flat = 0) or regrouped (flat = 1) */
static int make_tree(const uint8_t *lens, int flat, uint32_t *codes, int32_t *fd, ref_tree *t) {
    if (flat) {
        int rc = ref_flat_codes(lens, codes, fd);
        if (rc) return rc;
    } else {
        ref_canonical_codes(lens, codes);
        for (int s = 0; s < 256; s++) fd[s] = 0;
    }
    return build_tree(lens, codes, fd, t);
}

/* exported view of the tree for tests: depth, prefix, child ids (ordinary
   nodes), flat depth and symbol table (flat nodes, ftab[v * 256 + x]) */
int ref_tree_info_ex(const uint8_t *lens, int flat, int32_t *n_int, int32_t *depth, uint32_t *prefix, int32_t *child,
                     int32_t *fdepth, int32_t *ftab) {
    uint32_t codes[256]; int32_t fd[256];
    ref_tree *t = (ref_tree *)malloc(sizeof(ref_tree));
    if (!t) return REF_ERR_ARG;
    int rc = make_tree(lens, flat, codes, fd, t);
    if (rc) { free(t); return rc; }
    *n_int = t->n_int;
    for (int v = 0; v < t->n_int; v++) {
        depth[v] = t->depth[v]; prefix[v] = t->prefix[v];
        child[2 * v] = t->child[v][0]; child[2 * v + 1] = t->child[v][1];
        if (fdepth) fdepth[v] = t->flat[v];
        if (ftab) for (int x = 0; x < 256; x++) ftab[256 * v + x] = (t->flat[v] && x < (1 << t->flat[v])) ? t->ftab[v][x] : -1;
    }
    free(t);
    return REF_OK;
}

int ref_tree_info(const uint8_t *lens, int32_t *n_int, int32_t *depth, uint32_t *prefix, int32_t *child) {
    return ref_tree_info_ex(lens, 0, n_int, depth, prefix, child, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* 6a. ANS tables (Sec. 5.2: 50 static tables for skew 50..99 %, built */
/*     for bytes of i.i.d. bits; reading R5).                          */
/* ------------------------------------------------------------------ */
static const uint32_t BINOM8[9] = { 1, 8, 28, 56, 70, 56, 28, 8, 1 };

/* q[k] = frequency (out of M) of ONE byte with k one-bits under table t */
int ref_ans_class_freqs(int t, uint32_t *q) {
    if (t < 50 || t > 99) return REF_ERR_ARG;
    /* P(byte) * 100^8 = t^(8-k) * (100-t)^k exactly; M / 100^8 = 1 / D */
    const uint64_t D = 305175781250ull;          /* 10^16 / 2^15 */
    int64_t total = 0;
    for (int k = 0; k <= 8; k++) {
        uint64_t w = 1;
        for (int i = 0; i < 8 - k; i++) w *= (uint64_t)t;
        for (int i = 0; i < k; i++) w *= (uint64_t)(100 - t);
        uint64_t v = w / D;
        if (v == 0) v = 1;
        q[k] = (uint32_t)v;
        total += (int64_t)BINOM8[k] * (int64_t)v;
    }
    int64_t q0 = (int64_t)q[0] + ((int64_t)REF_ANS_M - total);
    if (q0 < 1) return REF_ERR_ARG;
    q[0] = (uint32_t)q0;
    return REF_OK;
}

/* per-byte frequency and cumulative start; bytes ordered by (popcount, value) */
static void ans_byte_table(int t, uint32_t *freq, uint32_t *cum) {
    uint32_t q[9];
    ref_ans_class_freqs(t, q);
    uint32_t c = 0;
    for (int k = 0; k <= 8; k++)
        for (int b = 0; b < 256; b++)
            if (popcount8((unsigned)b) == k) { freq[b] = q[k]; cum[b] = c; c += q[k]; }
}

/* expected ANS cost in bits per bitmap bit under table t for i.i.d. bits
   with P(0) = t/100 (the fse_H of Sec. 5.2), in double precision */
double ref_fse_h(int t) {
    uint32_t q[9];
    if (ref_ans_class_freqs(t, q)) return -1.0;
    double h = 0.0;
    for (int k = 0; k <= 8; k++) {
        double p = pow(t / 100.0, 8 - k) * pow((100 - t) / 100.0, k);
        h += (double)BINOM8[k] * p * log2((double)REF_ANS_M / (double)q[k]);
    }
    return h / 8.0;
}

int ref_fse_h_q16(int t) {
    double h = ref_fse_h(t);
    if (h < 0) return -1;
    return (int)floor(h * 65536.0 + 0.5);
}

/* ------------------------------------------------------------------ */
/* 6b. Interleaved rANS body of one bitmap (reading R5).               */
/*   body = u32 nwords[S], then per segment: W x u32 final states,     */
/*          nwords x u16 words (in decoder read order)                 */
/* ------------------------------------------------------------------ */
static uint32_t seg_count(uint32_t nbytes) { return (nbytes + REF_ANS_SEG - 1) / REF_ANS_SEG; }
static uint32_t seg_lanes(uint32_t seg_bytes) {
    uint32_t w = (seg_bytes + 511) / 512;
    if (w < 1) w = 1;
    if (w > 32) w = 32;
    return w;
}

int ref_rans_encode(const uint8_t *bytes, uint32_t nbytes, int t, uint8_t *body, uint64_t cap, uint64_t *body_bytes) {
    uint32_t freq[256], cum[256];
    if (t < 50 || t > 99 || nbytes == 0) return REF_ERR_ARG;
    ans_byte_table(t, freq, cum);
    uint32_t S = seg_count(nbytes);
    uint64_t pos = 4ull * S;
    uint16_t *stack = (uint16_t *)malloc(sizeof(uint16_t) * REF_ANS_SEG);
    if (!stack) return REF_ERR_ARG;
    for (uint32_t k = 0; k < S; k++) {
        uint32_t lo = k * REF_ANS_SEG, sb = nbytes - lo;
        if (sb > REF_ANS_SEG) sb = REF_ANS_SEG;
        uint32_t W = seg_lanes(sb);
        uint32_t x[32];
        for (uint32_t i = 0; i < W; i++) x[i] = REF_ANS_L;
        uint32_t nw = 0;
        /* encode in reverse; word emitted while encoding byte j is the word
           the decoder reads right after decoding byte j */
        for (int64_t j = (int64_t)sb - 1; j >= 0; j--) {
            uint32_t lane = (uint32_t)j % W;
            uint32_t b = bytes[lo + (uint32_t)j];
            uint64_t xs = x[lane];
            uint64_t xmax = ((uint64_t)(REF_ANS_L >> REF_ANS_SCALE) << 16) * freq[b];
            if (xs >= xmax) { stack[nw++] = (uint16_t)(xs & 0xFFFF); xs >>= 16; }
            xs = ((xs / freq[b]) << REF_ANS_SCALE) + (xs % freq[b]) + cum[b];
            x[lane] = (uint32_t)xs;
        }
        if (pos + 4ull * W + 2ull * nw > cap) { free(stack); return REF_ERR_CAPACITY; }
        put32(body + 4ull * k, nw);
        for (uint32_t i = 0; i < W; i++) put32(body + pos + 4ull * i, x[i]);
        pos += 4ull * W;
        for (uint32_t i = 0; i < nw; i++) put16(body + pos + 2ull * i, stack[nw - 1 - i]);
        pos += 2ull * nw;
    }
    free(stack);
    *body_bytes = pos;
    return REF_OK;
}

int ref_rans_decode(const uint8_t *body, uint64_t body_bytes, int t, uint8_t *bytes, uint32_t nbytes) {
    uint32_t freq[256], cum[256], slot2sym_start[257];
    int order[256];
    if (t < 50 || t > 99 || nbytes == 0) return REF_ERR_ARG;
    ans_byte_table(t, freq, cum);
    /* bytes in cumulative order, to look a slot up by linear search */
    { int n = 0; for (int k = 0; k <= 8; k++) for (int b = 0; b < 256; b++) if (popcount8((unsigned)b) == k) order[n++] = b; }
    for (int i = 0; i < 256; i++) slot2sym_start[i] = cum[order[i]];
    slot2sym_start[256] = REF_ANS_M;
    uint32_t S = seg_count(nbytes);
    uint64_t pos = 4ull * S;
    if (pos > body_bytes) return REF_ERR_CORRUPT;
    for (uint32_t k = 0; k < S; k++) {
        uint32_t lo = k * REF_ANS_SEG, sb = nbytes - lo;
        if (sb > REF_ANS_SEG) sb = REF_ANS_SEG;
        uint32_t W = seg_lanes(sb), nw = get32(body + 4ull * k);
        if (pos + 4ull * W + 2ull * nw > body_bytes) return REF_ERR_CORRUPT;
        uint32_t x[32];
        for (uint32_t i = 0; i < W; i++) x[i] = get32(body + pos + 4ull * i);
        pos += 4ull * W;
        const uint8_t *words = body + pos;
        uint32_t rd = 0;
        for (uint32_t i = 0; i < W; i++) if (x[i] < REF_ANS_L) return REF_ERR_CORRUPT;
        for (uint32_t j = 0; j < sb; j++) {
            uint32_t lane = j % W;
            uint32_t slot = x[lane] & (REF_ANS_M - 1);
            int r = 0;
            while (slot2sym_start[r + 1] <= slot) r++;
            uint32_t b = (uint32_t)order[r];
            x[lane] = freq[b] * (x[lane] >> REF_ANS_SCALE) + slot - cum[b];
            if (x[lane] < REF_ANS_L) {
                if (rd >= nw) return REF_ERR_CORRUPT;
                x[lane] = (x[lane] << 16) | get16(words + 2ull * rd);
                rd++;
            }
            bytes[lo + j] = (uint8_t)b;
        }
        if (rd != nw) return REF_ERR_CORRUPT;
        for (uint32_t i = 0; i < W; i++) if (x[i] != REF_ANS_L) return REF_ERR_CORRUPT;
        pos += 2ull * nw;
    }
    if (pos != body_bytes) return REF_ERR_CORRUPT;
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* 6b'. Skew analysis of Sec. 5.1: a node's benefit is the share of all */
/*      symbols that reach it times the bits entropy coding could save */
/*      per symbol there, 1 - H_b(skew).                               */
/* ------------------------------------------------------------------ */
double ref_binary_entropy(double p) {
    if (p <= 0.0 || p >= 1.0) return 0.0;
    return -(p * log2(p) + (1.0 - p) * log2(1.0 - p));
}

double ref_node_benefit(uint64_t n_v, uint64_t n1, uint64_t n_total) {
    if (n_v == 0 || n_total == 0) return 0.0;
    double skew = (double)(n1 > n_v - n1 ? n1 : n_v - n1) / (double)n_v;
    return ((double)n_v / (double)n_total) * (1.0 - ref_binary_entropy(skew));
}

/* ------------------------------------------------------------------ */
/* 6c. Selection rule of Sec. 5.2 (reading R6).  Returns the marker the */
/*     node gets if ANS is kept: 0 = not selected, else table id        */
/*     (t - 49) with bit 7 set for the XOR of the bitmap bytes.         */
/* ------------------------------------------------------------------ */
int ref_ans_select(uint64_t n_v, uint64_t n1, int depth, const ref_params *p) {
    if (!p->ans_enable || n_v == 0) return 0;
    uint64_t bytes = (n_v + 7) / 8;
    if (bytes < (uint64_t)p->ans_min_bytes) return 0;
    uint64_t n0 = n_v - n1, mx = n0 > n1 ? n0 : n1;
    /* skew = mx / n_v must be strictly higher than num/den */
    if (mx * (uint64_t)p->ans_skew_den <= (uint64_t)p->ans_skew_num * n_v) return 0;
    uint64_t t = (200 * mx + n_v) / (2 * n_v);      /* round half up of 100*skew */
    if (t < 50) t = 50;
    if (t > 99) t = 99;
    int fq = ref_fse_h_q16((int)t);
    /* (depth + fseH) / (depth + 1) strictly better (lower) than ratio */
    uint64_t lhs = ((uint64_t)depth * 65536u + (uint64_t)fq) * 100u;
    uint64_t rhs = (uint64_t)p->ans_ratio_pct * (uint64_t)(depth + 1) * 65536u;
    if (!(lhs < rhs)) return 0;
    int marker = (int)(t - 49);
    if (n1 > n0) marker |= 0x80;
    return marker;
}

/* ------------------------------------------------------------------ */
/* 7. Block record (App. D, adapted; reading R7)                        */
/*  0  u32 rec_bytes (multiple of 16)   4 u32 n                         */
/*  8  u16 n_int  10 u8 kind (0 empty, 1 constant, 2 coded)  11 u8 aux  */
/*  12 "PVC1" (canonical tree) or "PVC2" (regrouped tree, R10)          */
/*  kind 2: 16 lens[128] (symbol 2k low nibble of byte k)               */
/*          144 nv[n_int] u32, marker[n_int] u8, pad to 4,              */
/*          alen[n_sel] u32 (body bytes of each node with marker != 0), */
/*          raw bodies of marker-0 nodes, then bodies of the others,    */
/*          (a flat node's raw body is ceil(n_v * D / 8) bytes)         */
/*          zero pad to 16                                              */
/* ------------------------------------------------------------------ */
#define HDR_BYTES 16u
#define LENS_OFF 16u
#define NV_OFF 144u

static uint64_t pad16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

static void write_header(uint8_t *rec, uint32_t rec_bytes, uint32_t n, uint32_t n_int, uint32_t kind, uint32_t aux, int flat) {
    put32(rec, rec_bytes);
    put32(rec + 4, n);
    put16(rec + 8, n_int);
    rec[10] = (uint8_t)kind;
    rec[11] = (uint8_t)aux;
    rec[12] = 'P'; rec[13] = 'V'; rec[14] = 'C'; rec[15] = flat ? '2' : '1';
}

/* bits per element of node v's body: 1 for an ordinary node, D for a flat one */
static int node_bits(const ref_tree *t, int v) { return t->flat[v] ? t->flat[v] : 1; }

/* n_v of every node: the symbols whose code passes through it */
static void node_counts(const ref_tree *t, const uint8_t *lens, const uint32_t *codes, const int32_t *fd,
                        const uint32_t *hist, uint64_t *nv) {
    for (int v = 0; v < 256; v++) nv[v] = 0;
    for (int s = 0; s < 256; s++) {
        if (!lens[s]) continue;
        for (int d = 0; d < lens[s] - fd[s]; d++) nv[sym_node(t, lens, codes, s, d)] += hist[s];
        if (fd[s]) nv[sym_node(t, lens, codes, s, lens[s] - fd[s])] += hist[s];
    }
}

/* count of node v's right (bit 1) child, for the ANS rule */
static uint64_t right_count(const ref_tree *t, const uint64_t *nv, const uint32_t *hist, int v) {
    return t->child[v][1] >= 0 ? nv[t->child[v][1]] : hist[-t->child[v][1] - 1];
}

/* largest record the block can produce (every node stored raw) */
int ref_record_bound(const uint32_t *hist, const ref_params *p, uint64_t *bound) {
    uint8_t lens[256]; uint32_t codes[256]; int32_t fd[256];
    int K = 0;
    for (int s = 0; s < 256; s++) if (hist[s]) K++;
    if (K <= 1) { *bound = HDR_BYTES; return REF_OK; }
    int rc = ref_code_lengths(hist, p->max_len, lens);
    if (rc) return rc;
    ref_tree *t = (ref_tree *)malloc(sizeof(ref_tree));
    if (!t) return REF_ERR_ARG;
    rc = make_tree(lens, p->flat, codes, fd, t);
    if (rc) { free(t); return rc; }
    uint64_t nv[256];
    node_counts(t, lens, codes, fd, hist, nv);
    uint64_t sz = NV_OFF + 5ull * (uint64_t)t->n_int;
    sz = (sz + 3) & ~(uint64_t)3;
    int nsel_max = 0;
    for (int v = 0; v < t->n_int; v++) {
        sz += (nv[v] * (uint64_t)node_bits(t, v) + 7) / 8;
        if (!t->flat[v] && ref_ans_select(nv[v], right_count(t, nv, hist, v), t->depth[v], p)) nsel_max++;
    }
    sz += 4ull * (uint64_t)nsel_max;
    free(t);
    *bound = pad16(sz);
    return REF_OK;
}

int ref_encode_block(const uint8_t *x, uint64_t n, const ref_params *p, uint8_t *rec, uint64_t cap, uint64_t *rec_bytes) {
    uint32_t hist[256]; uint8_t lens[256]; uint32_t codes[256]; int32_t fd[256];
    if (n > 0xFFFFFFFFull) return REF_ERR_ARG;
    ref_histogram(x, n, hist);
    int K = 0, only = 0;
    for (int s = 0; s < 256; s++) if (hist[s]) { K++; only = s; }
    if (K <= 1) {
        if (cap < HDR_BYTES) return REF_ERR_CAPACITY;
        write_header(rec, HDR_BYTES, (uint32_t)n, 0, K == 0 ? 0u : 1u, K == 0 ? 0u : (uint32_t)only, p->flat);
        *rec_bytes = HDR_BYTES;
        return REF_OK;
    }
    int rc = ref_code_lengths(hist, p->max_len, lens);
    if (rc) return rc;
    ref_tree *t = (ref_tree *)malloc(sizeof(ref_tree));
    if (!t) return REF_ERR_ARG;
    rc = make_tree(lens, p->flat, codes, fd, t);
    if (rc) { free(t); return rc; }
    int V = t->n_int;

    /* 5. per-node bodies by the definition: in block order, append bit d of
          code(s) to the node named by its first d bits; a symbol that reaches
          a flat node appends its D-bit index there (value j at bits jD..) */
    uint64_t nv[256];
    node_counts(t, lens, codes, fd, hist, nv);
    uint8_t *bm[256];
    uint64_t cur[256];
    int node_of[256][16];
    for (int s = 0; s < 256; s++)
        if (lens[s]) for (int d = 0; d <= lens[s] - fd[s] && d < lens[s]; d++) node_of[s][d] = sym_node(t, lens, codes, s, d);
    for (int v = 0; v < V; v++) { bm[v] = (uint8_t *)calloc((size_t)((nv[v] * (uint64_t)node_bits(t, v) + 7) / 8) + 1, 1); cur[v] = 0; }
    for (uint64_t i = 0; i < n; i++) {
        int s = x[i];
        for (int d = 0; d < lens[s] - fd[s]; d++) {
            int v = node_of[s][d];
            uint32_t bit = (codes[s] >> (lens[s] - 1 - d)) & 1u;
            if (bit) bm[v][cur[v] >> 3] |= (uint8_t)(1u << (cur[v] & 7));
            cur[v]++;
        }
        if (fd[s]) {
            int v = node_of[s][lens[s] - fd[s]], D = fd[s];
            uint32_t xv = codes[s] & ((1u << D) - 1u);
            for (int k = 0; k < D; k++) {
                uint64_t pos = cur[v] * (uint64_t)D + (uint64_t)k;
                if ((xv >> k) & 1u) bm[v][pos >> 3] |= (uint8_t)(1u << (pos & 7));
            }
            cur[v]++;
        }
    }

    /* 6. selective ANS (ordinary nodes only) */
    int marker[256]; uint8_t *ans_body[256]; uint64_t ans_len[256];
    for (int v = 0; v < V; v++) {
        marker[v] = 0; ans_body[v] = NULL; ans_len[v] = 0;
        if (t->flat[v]) continue;
        int m = ref_ans_select(nv[v], right_count(t, nv, hist, v), t->depth[v], p);
        if (!m) continue;
        uint64_t raw = (nv[v] + 7) / 8;
        uint8_t *src = (uint8_t *)malloc((size_t)raw);
        for (uint64_t i = 0; i < raw; i++) src[i] = (m & 0x80) ? (uint8_t)(bm[v][i] ^ 0xFF) : bm[v][i];
        uint64_t bcap = 4 * ((raw + REF_ANS_SEG - 1) / REF_ANS_SEG) * 34 + 2 * raw + 64;
        uint8_t *body = (uint8_t *)malloc((size_t)bcap);
        uint64_t blen = 0;
        rc = ref_rans_encode(src, (uint32_t)raw, (m & 0x7F) + 49, body, bcap, &blen);
        free(src);
        if (rc) { free(body); for (int u = 0; u < V; u++) { free(bm[u]); free(ans_body[u]); } free(t); return rc; }
        if (blen >= raw) { free(body); marker[v] = (int)REF_MARK_RAW_SEL; ans_len[v] = raw; }
        else { marker[v] = m; ans_body[v] = body; ans_len[v] = blen; }
    }

    /* 7. serialise (marker[v] != 0: an ANS-coded or ANS-selected node) */
    int nsel = 0;
    for (int v = 0; v < V; v++) if (marker[v]) nsel++;
    uint64_t off = NV_OFF + 5ull * (uint64_t)V;
    off = (off + 3) & ~(uint64_t)3;
    uint64_t alen_off = off;
    off += 4ull * (uint64_t)nsel;
    uint64_t total = off;
    for (int v = 0; v < V; v++) total += marker[v] ? ans_len[v] : (nv[v] * (uint64_t)node_bits(t, v) + 7) / 8;
    total = pad16(total);
    if (total > cap || total > 0xFFFFFFFFull) {
        for (int v = 0; v < V; v++) { free(bm[v]); free(ans_body[v]); }
        free(t);
        return REF_ERR_CAPACITY;
    }
    memset(rec, 0, (size_t)total);
    write_header(rec, (uint32_t)total, (uint32_t)n, (uint32_t)V, 2, 0, p->flat);
    for (int k = 0; k < 128; k++) rec[LENS_OFF + k] = (uint8_t)(lens[2 * k] | (lens[2 * k + 1] << 4));
    for (int v = 0; v < V; v++) put32(rec + NV_OFF + 4ull * v, (uint32_t)nv[v]);
    for (int v = 0; v < V; v++) rec[NV_OFF + 4ull * V + v] = (uint8_t)(t->flat[v] ? REF_MARK_FLAT + (uint32_t)t->flat[v] : (uint32_t)marker[v]);
    { int k = 0; for (int v = 0; v < V; v++) if (marker[v]) put32(rec + alen_off + 4ull * (k++), (uint32_t)ans_len[v]); }
    for (int v = 0; v < V; v++) if (!marker[v]) {
        uint64_t b = (nv[v] * (uint64_t)node_bits(t, v) + 7) / 8;
        memcpy(rec + off, bm[v], (size_t)b); off += b;
    }
    for (int v = 0; v < V; v++) if (marker[v]) {
        if (ans_body[v]) memcpy(rec + off, ans_body[v], (size_t)ans_len[v]);
        else memcpy(rec + off, bm[v], (size_t)ans_len[v]);
        off += ans_len[v];
    }
    for (int v = 0; v < V; v++) { free(bm[v]); free(ans_body[v]); }
    free(t);
    *rec_bytes = total;
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* 8. Decode by the definition: for each output position walk from the */
/*    root, reading the next unread bit of each visited node (Listing 1 */
/*    on the pivoted layout of Sec. 2); a flat node gives its next      */
/*    D-bit index, the symbol of that index (Sec. 2.2.3).               */
/* ------------------------------------------------------------------ */
static int decode_coded(const uint8_t *rec, uint32_t rb, uint32_t n, uint32_t V, int flat, ref_tree *t, uint8_t *out) {
    uint8_t lens[256]; uint32_t codes[256]; int32_t fd[256];
    int K = 0;
    for (int k = 0; k < 128; k++) { lens[2 * k] = rec[LENS_OFF + k] & 15; lens[2 * k + 1] = rec[LENS_OFF + k] >> 4; }
    /* Kraft equality (a full tree) is required */
    uint64_t kraft = 0;
    for (int s = 0; s < 256; s++) if (lens[s]) { K++; kraft += 1ull << (15 - lens[s]); }
    if (K < 2 || kraft != (1ull << 15)) return REF_ERR_CORRUPT;
    if (make_tree(lens, flat, codes, fd, t) || t->n_int != (int)V) return REF_ERR_CORRUPT;
    uint64_t nv[256] = { 0 }; int marker[256];
    for (uint32_t v = 0; v < V; v++) {
        nv[v] = get32(rec + NV_OFF + 4ull * v);
        int m = rec[NV_OFF + 4ull * V + v];
        /* a flat node's marker names its depth; it is never ANS coded */
        if (t->flat[v]) {
            if (m != (int)REF_MARK_FLAT + t->flat[v]) return REF_ERR_CORRUPT;
            m = 0;
        }
        marker[v] = m;
    }
    if (nv[0] != n) return REF_ERR_CORRUPT;
    int nsel = 0;
    for (uint32_t v = 0; v < V; v++) {
        int m = marker[v];
        if (m) {
            nsel++;
            if (m != (int)REF_MARK_RAW_SEL && ((m & 0x7F) < 1 || (m & 0x7F) > 50)) return REF_ERR_CORRUPT;
        }
        /* every symbol below a node occurs at least once */
        if (nv[v] < (1ull << node_bits(t, (int)v))) return REF_ERR_CORRUPT;
        if (!t->flat[v]) for (int b = 0; b < 2; b++) if (t->child[v][b] >= 0 && nv[t->child[v][b]] > nv[v]) return REF_ERR_CORRUPT;
    }
    uint64_t off = NV_OFF + 5ull * V;
    off = (off + 3) & ~(uint64_t)3;
    uint64_t alen_off = off;
    off += 4ull * (uint64_t)nsel;
    if (off > rb) return REF_ERR_CORRUPT;
    /* bodies: raw ones point into the record, ANS ones are decoded */
    const uint8_t *bm[256]; uint8_t *owned[256];
    uint64_t nbits[256];
    int k = 0;
    for (uint32_t v = 0; v < V; v++) { owned[v] = NULL; nbits[v] = nv[v] * (uint64_t)node_bits(t, (int)v); }
    uint64_t alen[256];
    for (uint32_t v = 0; v < V; v++) alen[v] = marker[v] ? get32(rec + alen_off + 4ull * (k++)) : 0;
    int rc = REF_OK;
    for (uint32_t v = 0; v < V; v++) if (!marker[v]) {
        uint64_t b = (nbits[v] + 7) / 8;
        if (off + b > rb) { rc = REF_ERR_CORRUPT; goto done; }
        bm[v] = rec + off; off += b;
    }
    for (uint32_t v = 0; v < V; v++) if (marker[v]) {
        uint64_t raw = (nv[v] + 7) / 8;
        if (off + alen[v] > rb) { rc = REF_ERR_CORRUPT; goto done; }
        if (marker[v] == (int)REF_MARK_RAW_SEL) {
            if (alen[v] != raw) { rc = REF_ERR_CORRUPT; goto done; }
            bm[v] = rec + off;
        } else {
            owned[v] = (uint8_t *)malloc((size_t)raw);
            if (ref_rans_decode(rec + off, alen[v], (marker[v] & 0x7F) + 49, owned[v], (uint32_t)raw)) { rc = REF_ERR_CORRUPT; goto done; }
            if (marker[v] & 0x80) for (uint64_t i = 0; i < raw; i++) owned[v][i] ^= 0xFF;
            bm[v] = owned[v];
        }
        off += alen[v];
    }
    if (pad16(off) != rb) { rc = REF_ERR_CORRUPT; goto done; }
    for (uint64_t i = off; i < rb; i++) if (rec[i]) { rc = REF_ERR_CORRUPT; goto done; }
    {
        uint64_t cursor[256];
        for (uint32_t v = 0; v < V; v++) cursor[v] = 0;
        for (uint32_t i = 0; i < n; i++) {
            int v = 0;
            for (;;) {
                if (cursor[v] >= nv[v]) { rc = REF_ERR_CORRUPT; goto done; }
                uint64_t j = cursor[v]++;
                if (t->flat[v]) {
                    int D = t->flat[v];
                    uint32_t xv = 0;
                    for (int q = 0; q < D; q++) {
                        uint64_t pos = j * (uint64_t)D + (uint64_t)q;
                        xv |= (uint32_t)((bm[v][pos >> 3] >> (pos & 7)) & 1u) << q;
                    }
                    out[i] = t->ftab[v][xv];
                    break;
                }
                int bit = (bm[v][j >> 3] >> (j & 7)) & 1;
                int c = t->child[v][bit];
                if (c < 0) { out[i] = (uint8_t)(-c - 1); break; }
                v = c;
            }
        }
        for (uint32_t v = 0; v < V; v++) {
            if (cursor[v] != nv[v]) { rc = REF_ERR_CORRUPT; goto done; }
            /* pad bits of the last byte are zero */
            if (nbits[v] & 7) { if (bm[v][nbits[v] >> 3] >> (nbits[v] & 7)) { rc = REF_ERR_CORRUPT; goto done; } }
        }
    }
done:
    for (uint32_t v = 0; v < V; v++) free(owned[v]);
    return rc;
}

int ref_decode_block(const uint8_t *rec, uint64_t avail, uint8_t *out, uint64_t cap, uint64_t *n_out) {
    if (avail < HDR_BYTES) return REF_ERR_CORRUPT;
    uint32_t rb = get32(rec), n = get32(rec + 4), V = get16(rec + 8), kind = rec[10], aux = rec[11];
    if (rec[12] != 'P' || rec[13] != 'V' || rec[14] != 'C' || (rec[15] != '1' && rec[15] != '2')) return REF_ERR_CORRUPT;
    int flat = rec[15] == '2';
    if (rb < HDR_BYTES || (rb & 15u) || rb > avail) return REF_ERR_CORRUPT;
    if (n > cap) return REF_ERR_CAPACITY;
    *n_out = n;
    if (kind == 0) { if (n != 0 || V != 0 || aux != 0 || rb != HDR_BYTES) return REF_ERR_CORRUPT; return REF_OK; }
    if (kind == 1) {
        if (n == 0 || V != 0 || rb != HDR_BYTES) return REF_ERR_CORRUPT;
        for (uint32_t i = 0; i < n; i++) out[i] = (uint8_t)aux;
        return REF_OK;
    }
    if (kind != 2 || aux != 0 || n == 0 || V < 1 || V > 255) return REF_ERR_CORRUPT;
    if (rb < NV_OFF + 5ull * V) return REF_ERR_CORRUPT;
    ref_tree *t = (ref_tree *)malloc(sizeof(ref_tree));
    if (!t) return REF_ERR_ARG;
    int rc = decode_coded(rec, rb, n, V, flat, t, out);
    free(t);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Batch helpers (many blocks, caller offsets), used by tests and the  */
/* CPU baseline.  Records go to rec + rec_off[b]; rec_bytes[b] out.    */
/* ------------------------------------------------------------------ */
int ref_encode_batch(const uint8_t *x, const uint64_t *blk_off, int nblk, const ref_params *p,
                     uint8_t *rec, const uint64_t *rec_off, const uint64_t *rec_cap, uint64_t *rec_bytes) {
    for (int b = 0; b < nblk; b++) {
        int rc = ref_encode_block(x + blk_off[b], blk_off[b + 1] - blk_off[b], p, rec + rec_off[b], rec_cap[b], &rec_bytes[b]);
        if (rc) return rc;
    }
    return REF_OK;
}

int ref_decode_batch(const uint8_t *rec, const uint64_t *rec_off, const uint64_t *rec_avail, int nblk,
                     uint8_t *out, const uint64_t *out_off, int32_t *status) {
    int bad = 0;
    for (int b = 0; b < nblk; b++) {
        uint64_t n = 0;
        status[b] = ref_decode_block(rec + rec_off[b], rec_avail[b], out + out_off[b], out_off[b + 1] - out_off[b], &n);
        if (!status[b] && n != out_off[b + 1] - out_off[b]) status[b] = REF_ERR_CORRUPT;
        if (status[b]) bad++;
    }
    return bad ? REF_ERR_CORRUPT : REF_OK;
}

/* ------------------------------------------------------------------------ */
/* PivCo-Golomb (App. G).                                                    */
/*                                                                          */
/* Reading: App. G applies pivoted coding to Golomb coding with a LIST of    */
/* bitmaps in place of a tree.  Here the Golomb parameter is 1, i.e. the     */
/* unary code: value v is written as v "continue" bits then one "stop" bit,   */
/* and stop = 1 (App. G: a 1 bit yields output 0x00, a 0 bit the child's      */
/* value plus 1).  Pivoted: bitmap j holds, in sequence order, the j-th code  */
/* bit of every value with at least j+1 code bits, i.e. of every v >= j: 1    */
/* if v == j, 0 if v > j.  There are m = (largest value) + 1 bitmaps.         */
/*                                                                          */
/* Record (byte-aligned like App. D; u32 widths as in the PivCo record):      */
/*    0 u32 rec_bytes (multiple of 16)   4 u32 n   8 u16 m   10 u8 kind = 4   */
/*   11 u8 0   12 "PVG1"   16 u32 n_j[m] (values >= j; n_0 = n)               */
/*   then the bitmaps B_0 .. B_{m-1}, ceil(n_j / 8) bytes each, back to back, */
/*   bit i of B_j in byte i >> 3 at bit (i & 7), pad bits 0; zero pad to 16.  */
/* An empty sequence is a 16-byte record with n = m = 0.                     */
/* ------------------------------------------------------------------------ */
#define REF_GOLOMB_KIND 4u

int ref_golomb_bound(const uint8_t *x, uint64_t n, uint64_t *bound) {
    if (!bound || n > 0xFFFFFFFFull || (n && !x)) return REF_ERR_ARG;
    uint64_t cnt[257];
    memset(cnt, 0, sizeof cnt);
    int m = 0;
    for (uint64_t i = 0; i < n; i++) { cnt[x[i]]++; if ((int)x[i] + 1 > m) m = (int)x[i] + 1; }
    /* n_j = values >= j: a suffix sum of the counts */
    uint64_t ge = 0, bytes = 16 + 4ull * (uint64_t)m;
    for (int j = 255; j >= 0; j--) { ge += cnt[j]; if (j < m) bytes += (ge + 7) / 8; }
    *bound = pad16(bytes);
    return REF_OK;
}

int ref_golomb_encode(const uint8_t *x, uint64_t n, uint8_t *rec, uint64_t cap, uint64_t *rec_bytes) {
    uint64_t size = 0;
    int rc = ref_golomb_bound(x, n, &size);
    if (rc != REF_OK) return rc;
    if (!rec || cap < size) return REF_ERR_CAPACITY;
    memset(rec, 0, size);
    int m = 0;
    for (uint64_t i = 0; i < n; i++) if ((int)x[i] + 1 > m) m = (int)x[i] + 1;
    put32(rec, (uint32_t)size);
    put32(rec + 4, (uint32_t)n);
    put16(rec + 8, (uint32_t)m);
    rec[10] = (uint8_t)REF_GOLOMB_KIND;
    rec[11] = 0;
    memcpy(rec + 12, "PVG1", 4);
    /* n_j and the bitmap starts */
    uint64_t nj[256], start[256], off = 16 + 4ull * (uint64_t)m;
    for (int j = 0; j < m; j++) {
        nj[j] = 0;
        for (uint64_t i = 0; i < n; i++) nj[j] += x[i] >= j;
        put32(rec + 16 + 4 * j, (uint32_t)nj[j]);
        start[j] = off;
        off += (nj[j] + 7) / 8;
    }
    /* value by value, code bit by code bit: bit j of value v goes to the next
       free position of bitmap j */
    uint64_t cur[256];
    memset(cur, 0, sizeof cur);
    for (uint64_t i = 0; i < n; i++) {
        for (int j = 0; j <= x[i]; j++) {
            const uint64_t pos = cur[j]++;
            if (j == x[i]) rec[start[j] + (pos >> 3)] |= (uint8_t)(1u << (pos & 7));
        }
    }
    if (rec_bytes) *rec_bytes = size;
    return REF_OK;
}

/* Decode by the definition: for each output, read bitmaps 0, 1, ... at their
   own cursors until a stop bit; the value is the number of continue bits. */
int ref_golomb_decode(const uint8_t *rec, uint64_t avail, uint8_t *out, uint64_t cap, uint64_t *n_out) {
    if (!rec || avail < 16) return REF_ERR_CORRUPT;
    const uint32_t size = get32(rec), n = get32(rec + 4), m = get16(rec + 8);
    if (memcmp(rec + 12, "PVG1", 4) != 0 || rec[10] != REF_GOLOMB_KIND || rec[11] != 0 || size % 16 || size > avail ||
        m > 256 || (n == 0) != (m == 0) || 16ull + 4ull * m > size)
        return REF_ERR_CORRUPT;
    if (n_out) *n_out = n;
    if (n > cap || (n && !out)) return REF_ERR_CAPACITY;
    uint64_t nj[256], start[256], off = 16 + 4ull * m;
    for (uint32_t j = 0; j < m; j++) {
        nj[j] = get32(rec + 16 + 4 * j);
        if ((j == 0 && nj[j] != n) || (j && nj[j] > nj[j - 1])) return REF_ERR_CORRUPT;
        start[j] = off;
        off += (nj[j] + 7) / 8;
    }
    if (pad16(off) != size) return REF_ERR_CORRUPT;
    uint64_t cur[256];
    memset(cur, 0, sizeof cur);
    for (uint32_t i = 0; i < n; i++) {
        uint32_t j = 0;
        for (;;) {
            if (j >= m || cur[j] >= nj[j]) return REF_ERR_CORRUPT;
            const uint64_t pos = cur[j]++;
            if ((rec[start[j] + (pos >> 3)] >> (pos & 7)) & 1u) break;
            j++;
        }
        out[i] = (uint8_t)j;
    }
    /* every bitmap read exactly to its end; pad bits zero */
    for (uint32_t j = 0; j < m; j++) {
        if (cur[j] != nj[j]) return REF_ERR_CORRUPT;
        if ((nj[j] & 7) && (rec[start[j] + (nj[j] >> 3)] >> (nj[j] & 7))) return REF_ERR_CORRUPT;
    }
    for (uint64_t i = off; i < size; i++) if (rec[i]) return REF_ERR_CORRUPT;
    return REF_OK;
}
