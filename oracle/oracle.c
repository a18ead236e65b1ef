/*
 * CPU oracle: approximate 1-Wasserstein distance between persistence diagrams
 * by graph sparsification (Dey & Zhang, "Approximating 1-Wasserstein Distance
 * between Persistence Diagrams by Graph Sparsification").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, sequential, obviously correct
 * restatement of the method that the CUDA library is checked against.  It
 * shares no code, header, table or constant generator with the CUDA library.
 * Only tests/, the smoke entry point and the benchmark's CPU-baseline leg may
 * load it; the product path never does.
 *
 * Everything is exact integer arithmetic on coordinates quantised to a
 * power-of-two quantum q = 2^-k, with every ground cost rounded UP to a whole
 * quantum (so rounded costs still obey the triangle inequality), except
 * orc_w1_exact(), which is the exact FP64 W1 on the unquantised points.
 *
 * Paper map (section / equation / algorithm):
 *   orc_quantize ........ points of a diagram (Problem Formulation; b != d)
 *   orc_condense0 ....... 0-condensation: the node sets Â, B̂ of G(A,B)
 *   orc_cost, orc_cdiag . l2 ground metric and distance to the diagonal (Problem Formulation)
 *   orc_rwmd ............ RWMD lower bound, Algorithm 1, including the arc to ā
 *                         that the relaxed min-cost flow contains
 *   orc_s_from_eps ...... the tighter bound 1+eps = (1+4/s+4/(s-2))(1+8/(s-4)) (Experiments)
 *   orc_delta_params .... Algorithm 2's eps and delta; k = 0.99 lattice, (1-k)/2 shift
 *   orc_condense_delta .. Algorithm 2: snap to the common lattice, aggregate supplies, perturb
 *   orc_radix_tree ...... hierarchical decomposition for the WSPD (a compressed quadtree
 *                         over Morton order stands in for the split tree)
 *   orc_wspd ............ s-WSPD (well-separated definition; Algorithms 6-8), biarcs
 *   orc_build_network ... diagonal arcs (Algorithm 9) + CSR "static graph" (Appendix)
 *   orc_ns_int/_dbl ..... network simplex with block search pivoting, run to optimality
 *   orc_w1_exact ........ exact W1 by min-cost flow on G(A,B) (Proposition: matching iff flow)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------- */
/* Exact integer square roots.                                                */
/* ------------------------------------------------------------------------- */

/* floor(sqrt(v)), digit-by-digit (base 4) method. */
uint64_t orc_isqrt(uint64_t v) {
    uint64_t res = 0, bit = (uint64_t)1 << 62;
    while (bit > v) bit >>= 2;
    while (bit) {
        if (v >= res + bit) {
            v -= res + bit;
            res = (res >> 1) + bit;
        } else {
            res >>= 1;
        }
        bit >>= 2;
    }
    return res;
}

/* smallest r with r*r >= v */
uint64_t orc_ceil_sqrt(uint64_t v) {
    uint64_t r = orc_isqrt(v);
    return (r * r < v) ? r + 1 : r;
}

/* l2 ground cost between two quantised points, rounded up to a whole quantum. */
int64_t orc_cost(int64_t x1, int64_t y1, int64_t x2, int64_t y2) {
    int64_t dx = x1 - x2, dy = y1 - y2;
    uint64_t d2 = (uint64_t)(dx * dx) + (uint64_t)(dy * dy);
    return (int64_t)orc_ceil_sqrt(d2);
}

/* l2 distance of (x,y) to the diagonal y = x, |y - x| / sqrt(2), rounded up:
 * the smallest c with 2 c^2 >= t^2, i.e. c = ceil_sqrt(ceil(t^2 / 2)). */
int64_t orc_cdiag(int64_t x, int64_t y) {
    int64_t t = y - x;
    if (t < 0) t = -t;
    uint64_t t2 = (uint64_t)t * (uint64_t)t;
    return (int64_t)orc_ceil_sqrt((t2 + 1) / 2);
}

/* Cost of destroying a unit at (x, y) (arc u -> ā) or creating one there
 * (b̄ -> v): the distance to the diagonal for persistence diagrams (kappa 1,
 * tau 0).  The Conclusion's unbalanced optimal transport on R^2 reassigns
 * these arcs' costs to creation / destruction costs; here kappa * d_diag + tau
 * with kappa in {0, 1} and tau >= 0 quanta (kappa 0: a constant cost). */
int64_t orc_cmake(int64_t x, int64_t y, int64_t kappa, int64_t tau) {
    return (kappa ? orc_cdiag(x, y) : 0) + tau;
}

static int64_t floordiv(int64_t a, int64_t b) { /* b > 0 */
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q--;
    return q;
}

/* ------------------------------------------------------------------------- */
/* Quantisation of a diagram.                                                */
/* ------------------------------------------------------------------------- */

#define ORC_COORD_LIMIT ((int64_t)1 << 29)

/* bd: interleaved (b, d) pairs, n of them; dtype 0 = float32, 1 = uint8.
 * X = rint(b * 2^k), Y = rint(d * 2^k) (round half to even; exact for uint8).
 * Points with X == Y lie on the diagonal and are dropped.  Returns the number
 * of points kept, or -1 if a coordinate is not finite or |X|,|Y| >= 2^29. */
int64_t orc_quantize(const void* bd, int64_t n, int dtype, int k, int32_t* X, int32_t* Y) {
    int64_t kept = 0;
    double scale = ldexp(1.0, k);
    for (int64_t i = 0; i < n; i++) {
        int64_t qx, qy;
        if (dtype == 0) {
            const float* f = (const float*)bd;
            double b = (double)f[2 * i], d = (double)f[2 * i + 1];
            if (!isfinite(b) || !isfinite(d)) return -1;
            double vb = rint(b * scale), vd = rint(d * scale);
            if (fabs(vb) >= (double)ORC_COORD_LIMIT || fabs(vd) >= (double)ORC_COORD_LIMIT) return -1;
            qx = (int64_t)vb;
            qy = (int64_t)vd;
        } else {
            const uint8_t* u = (const uint8_t*)bd;
            qx = (int64_t)u[2 * i] << k;
            qy = (int64_t)u[2 * i + 1] << k;
            if (qx >= ORC_COORD_LIMIT || qy >= ORC_COORD_LIMIT) return -1;
        }
        if (qx == qy) continue;
        X[kept] = (int32_t)qx;
        Y[kept] = (int32_t)qy;
        kept++;
    }
    return kept;
}

/* ------------------------------------------------------------------------- */
/* 0-condensation: coincident points of one diagram become one node.          */
/* ------------------------------------------------------------------------- */

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

static uint64_t pack_xy(int64_t x, int64_t y) { /* order-preserving for |x|,|y| < 2^31 */
    return ((uint64_t)(x + ((int64_t)1 << 31)) << 32) | (uint64_t)(y + ((int64_t)1 << 31));
}

/* Nodes come out sorted by (X, Y).  Returns the number of nodes. */
int64_t orc_condense0(const int32_t* X, const int32_t* Y, int64_t n,
                      int32_t* UX, int32_t* UY, int64_t* cnt) {
    if (n == 0) return 0;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * n);
    for (int64_t i = 0; i < n; i++) key[i] = pack_xy(X[i], Y[i]);
    qsort(key, n, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        if (i == 0 || key[i] != key[i - 1]) {
            UX[m] = (int32_t)((int64_t)(key[i] >> 32) - ((int64_t)1 << 31));
            UY[m] = (int32_t)((int64_t)(key[i] & 0xffffffffu) - ((int64_t)1 << 31));
            cnt[m] = 0;
            m++;
        }
        cnt[m - 1]++;
    }
    free(key);
    return m;
}

/* ------------------------------------------------------------------------- */
/* RWMD lower bound (Algorithm 1).                                            */
/* ------------------------------------------------------------------------- */

/* One side of Algorithm 1: every unit at node u of P is sent to the cheapest
 * node of Q or, as the relaxed min-cost flow also allows, to the diagonal
 * node (cost d_diag(u), or the destruction cost of orc_cmake).
 * min_v ceil(sqrt(d2)) = ceil(sqrt(min_v d2)).                              */
static int64_t rwmd_side(const int32_t* PX, const int32_t* PY, const int64_t* Pc, int64_t nP,
                         const int32_t* QX, const int32_t* QY, int64_t nQ, int64_t kappa, int64_t tau) {
    int64_t L = 0;
    for (int64_t u = 0; u < nP; u++) {
        int64_t best = orc_cmake(PX[u], PY[u], kappa, tau);
        if (nQ > 0) {
            uint64_t bd2 = UINT64_MAX;
            for (int64_t v = 0; v < nQ; v++) {
                int64_t dx = (int64_t)PX[u] - QX[v], dy = (int64_t)PY[u] - QY[v];
                uint64_t d2 = (uint64_t)(dx * dx) + (uint64_t)(dy * dy);
                if (d2 < bd2) bd2 = d2;
            }
            int64_t c = (int64_t)orc_ceil_sqrt(bd2);
            if (c < best) best = c;
        }
        L += Pc[u] * best;
    }
    return L;
}

/* L[0] = L_A, L[1] = L_B, L[2] = max(L_A, L_B), all in quanta. */
void orc_rwmd(const int32_t* AX, const int32_t* AY, const int64_t* Ac, int64_t nA,
              const int32_t* BX, const int32_t* BY, const int64_t* Bc, int64_t nB, int64_t kappa, int64_t tau,
              int64_t* L) {
    L[0] = rwmd_side(AX, AY, Ac, nA, BX, BY, nB, kappa, tau);
    L[1] = rwmd_side(BX, BY, Bc, nB, AX, AY, nA, kappa, tau);
    L[2] = L[0] > L[1] ? L[0] : L[1];
}

/* ------------------------------------------------------------------------- */
/* eps -> s, delta (Algorithm 2; tighter bound from the Experiments).        */
/* ------------------------------------------------------------------------- */

double orc_bound(int64_t s) {
    double sd = (double)s;
    return (1.0 + 4.0 / sd + 4.0 / (sd - 2.0)) * (1.0 + 8.0 / (sd - 4.0));
}

/* smallest integer s >= 13 with (1 + 4/s + 4/(s-2)) (1 + 8/(s-4)) <= 1 + eps */
int64_t orc_s_from_eps(double eps) {
    if (!(eps > 0.0)) return -1;
    for (int64_t s = 13; s < ((int64_t)1 << 40); s++)
        if (orc_bound(s) <= 1.0 + eps) return s;
    return -1;
}

/* eps_c = 8/(s-4) for s >= 12, else 1 (Algorithm 2). */
double orc_eps_c(int64_t s) { return s >= 12 ? 8.0 / (double)(s - 4) : 1.0; }

#define ORC_G_MAX ((int64_t)1 << 28)

/* L_lo = max(L_A - F_A, L_B - F_B, 0) is a lower bound on the real-valued
 * RWMD (each rounded-up unit cost exceeds its real cost by < 1 quantum), so
 * delta = 2 eps_c L_lo / (sqrt(2) (|A~| + |B~|)) keeps Proposition
 * (delta-condensation) valid.  Lattice spacing G = max(1, floor(0.99 delta)),
 * shift bound P = floor(0.005 delta) (k = 0.99, shift (1-k) delta / 2),
 * clamped so that 2P < G and G <= 2^28. */
void orc_delta_params(int64_t LA, int64_t LB, int64_t FA, int64_t FB, int64_t s,
                      double* delta_out, int64_t* G_out, int64_t* P_out) {
    int64_t Llo = LA - FA;
    if (LB - FB > Llo) Llo = LB - FB;
    if (Llo < 0) Llo = 0;
    double eps_c = orc_eps_c(s);
    double delta = 0.0;
    if (FA + FB > 0) delta = 2.0 * eps_c * (double)Llo / (sqrt(2.0) * (double)(FA + FB));
    double g = floor(0.99 * delta);
    int64_t G = (g >= (double)ORC_G_MAX) ? ORC_G_MAX : (int64_t)g;
    if (G < 1) G = 1;
    double p = floor(0.005 * delta);
    int64_t P = (p >= (double)ORC_G_MAX) ? ORC_G_MAX : (int64_t)p;
    if (2 * P >= G) P = (G - 1) / 2;
    *delta_out = delta;
    *G_out = G;
    *P_out = P;
}

/* ------------------------------------------------------------------------- */
/* delta-condensation (Algorithm 2) and Morton order.                        */
/* ------------------------------------------------------------------------- */

/* SplitMix64 output finaliser (Steele, Lea & Flood 2014). */
uint64_t orc_mix64(uint64_t z);
static uint64_t mix64(uint64_t z) { return orc_mix64(z); }
uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The random shift of a condensed point, a pure function of (seed, cell):
 * two rounds of the finaliser give independent offsets in [-P, P]. */
void orc_perturb(uint64_t seed, int64_t cx, int64_t cy, int64_t P, int64_t* dx, int64_t* dy) {
    if (P <= 0) {
        *dx = 0;
        *dy = 0;
        return;
    }
    uint64_t h1 = mix64(seed ^ ((uint64_t)cx * 0x9E3779B97F4A7C15ULL) ^ ((uint64_t)cy * 0xC2B2AE3D27D4EB4FULL));
    uint64_t h2 = mix64(h1 + 0x9E3779B97F4A7C15ULL);
    uint64_t span = (uint64_t)(2 * P + 1);
    *dx = (int64_t)(h1 % span) - P;
    *dy = (int64_t)(h2 % span) - P;
}

static uint64_t spread_bits(uint32_t v) {
    uint64_t r = 0;
    for (int i = 0; i < 32; i++) r |= (uint64_t)((v >> i) & 1u) << (2 * i);
    return r;
}

/* Morton code: bit i of x goes to bit 2i, bit i of y to bit 2i+1. */
uint64_t orc_morton(uint32_t x, uint32_t y) { return spread_bits(x) | (spread_bits(y) << 1); }

typedef struct {
    int64_t cx, cy, ca, cb;
} cellrec_t;

static int cmp_cell(const void* a, const void* b) {
    const cellrec_t* p = (const cellrec_t*)a;
    const cellrec_t* q = (const cellrec_t*)b;
    if (p->cx != q->cx) return p->cx < q->cx ? -1 : 1;
    if (p->cy != q->cy) return p->cy < q->cy ? -1 : 1;
    return 0;
}

typedef struct {
    uint64_t code;
    int32_t x, y;
    int64_t ca, cb;
} noderec_t;

static int cmp_node(const void* a, const void* b) {
    uint64_t x = ((const noderec_t*)a)->code, y = ((const noderec_t*)b)->code;
    return (x > y) - (x < y);
}

/* Snap every node of Â and B̂ to the common lattice G*Z x G*Z (round half
 * up: cell = floor((2X + G) / (2G))), aggregate the multiplicities per cell,
 * place each cell's node at G*cell + shift(seed, cell), and order the nodes by
 * the Morton code of (X - min X, Y - min Y).  Returns N, the number of nodes;
 * cntA/cntB are the aggregated multiplicities of A and B at each node. */
int64_t orc_condense_delta(const int32_t* AX, const int32_t* AY, const int64_t* Ac, int64_t nA,
                           const int32_t* BX, const int32_t* BY, const int64_t* Bc, int64_t nB,
                           int64_t G, int64_t P, uint64_t seed,
                           int32_t* X, int32_t* Y, int64_t* cntA, int64_t* cntB, uint64_t* code) {
    int64_t n = nA + nB;
    if (n == 0) return 0;
    cellrec_t* c = (cellrec_t*)malloc(sizeof(cellrec_t) * n);
    for (int64_t i = 0; i < nA; i++) {
        c[i].cx = floordiv(2 * (int64_t)AX[i] + G, 2 * G);
        c[i].cy = floordiv(2 * (int64_t)AY[i] + G, 2 * G);
        c[i].ca = Ac[i];
        c[i].cb = 0;
    }
    for (int64_t i = 0; i < nB; i++) {
        c[nA + i].cx = floordiv(2 * (int64_t)BX[i] + G, 2 * G);
        c[nA + i].cy = floordiv(2 * (int64_t)BY[i] + G, 2 * G);
        c[nA + i].ca = 0;
        c[nA + i].cb = Bc[i];
    }
    qsort(c, n, sizeof(cellrec_t), cmp_cell);
    noderec_t* nd = (noderec_t*)malloc(sizeof(noderec_t) * n);
    int64_t N = 0;
    for (int64_t i = 0; i < n; i++) {
        if (i == 0 || cmp_cell(&c[i], &c[i - 1]) != 0) {
            int64_t dx, dy;
            orc_perturb(seed, c[i].cx, c[i].cy, P, &dx, &dy);
            nd[N].x = (int32_t)(G * c[i].cx + dx);
            nd[N].y = (int32_t)(G * c[i].cy + dy);
            nd[N].ca = 0;
            nd[N].cb = 0;
            N++;
        }
        nd[N - 1].ca += c[i].ca;
        nd[N - 1].cb += c[i].cb;
    }
    int64_t mnx = nd[0].x, mny = nd[0].y;
    for (int64_t i = 1; i < N; i++) {
        if (nd[i].x < mnx) mnx = nd[i].x;
        if (nd[i].y < mny) mny = nd[i].y;
    }
    for (int64_t i = 0; i < N; i++)
        nd[i].code = orc_morton((uint32_t)(nd[i].x - mnx), (uint32_t)(nd[i].y - mny));
    qsort(nd, N, sizeof(noderec_t), cmp_node);
    for (int64_t i = 0; i < N; i++) {
        X[i] = nd[i].x;
        Y[i] = nd[i].y;
        cntA[i] = nd[i].ca;
        cntB[i] = nd[i].cb;
        code[i] = nd[i].code;
    }
    free(c);
    free(nd);
    return N;
}

/* ------------------------------------------------------------------------- */
/* Hierarchical decomposition: binary radix tree over sorted Morton codes.    */
/* ------------------------------------------------------------------------- */

/* Internal node w covers the leaf range [lo, hi] (lo < hi).  Its split is the
 * last index whose code has a 0 at the highest bit where code[lo] and
 * code[hi] differ.  Numbering: the root is internal node 0; a child covering
 * [lo, split] (if internal) is numbered split, a child covering
 * [split+1, hi] (if internal) is numbered split+1.  Children are encoded as
 * c >= 0 for internal node c and c < 0 for leaf ~c.  For every internal node
 * the tight bounding box bb = (minX, maxX, minY, maxY) and the leftmost member
 * (min X, then min Y) are computed directly from its range.  Needs N >= 2. */
void orc_radix_tree(int64_t N, const uint64_t* code, const int32_t* X, const int32_t* Y,
                    int32_t* left, int32_t* right, int32_t* lo_out, int32_t* hi_out,
                    int32_t* bb, int32_t* rep) {
    if (N < 2) return;
    int64_t* stk = (int64_t*)malloc(sizeof(int64_t) * 3 * (N + 1));
    int64_t sp = 0;
    stk[sp++] = 0;
    stk[sp++] = N - 1;
    stk[sp++] = 0;
    while (sp > 0) {
        int64_t w = stk[--sp], hi = stk[--sp], lo = stk[--sp];
        uint64_t diff = code[lo] ^ code[hi];
        int d = 63;
        while (!((diff >> d) & 1u)) d--;
        int64_t split = lo;
        for (int64_t i = lo; i < hi; i++)
            if (!((code[i] >> d) & 1u)) split = i;
        lo_out[w] = (int32_t)lo;
        hi_out[w] = (int32_t)hi;
        left[w] = (split == lo) ? (int32_t)~lo : (int32_t)split;
        right[w] = (split + 1 == hi) ? (int32_t)~hi : (int32_t)(split + 1);
        int32_t mnx = X[lo], mxx = X[lo], mny = Y[lo], mxy = Y[lo];
        int64_t r = lo;
        for (int64_t i = lo; i <= hi; i++) {
            if (X[i] < mnx) mnx = X[i];
            if (X[i] > mxx) mxx = X[i];
            if (Y[i] < mny) mny = Y[i];
            if (Y[i] > mxy) mxy = Y[i];
            if (X[i] < X[r] || (X[i] == X[r] && Y[i] < Y[r])) r = i;
        }
        bb[4 * w + 0] = mnx;
        bb[4 * w + 1] = mxx;
        bb[4 * w + 2] = mny;
        bb[4 * w + 3] = mxy;
        rep[w] = (int32_t)r;
        if (split != lo) {
            stk[sp++] = lo;
            stk[sp++] = split;
            stk[sp++] = split;
        }
        if (split + 1 != hi) {
            stk[sp++] = split + 1;
            stk[sp++] = hi;
            stk[sp++] = split + 1;
        }
    }
    free(stk);
}

/* ------------------------------------------------------------------------- */
/* The paper's split tree (WSPD section): take the bounding box of a point    */
/* set, cut its longest side in the middle, recurse until single points.      */
/* ------------------------------------------------------------------------- */

/* Split tree over the N nodes (X, Y).  A set of two or more points is cut at
 * the middle of the longest side of its tight bounding box (the x side when
 * the sides are equal): a point goes left when twice its coordinate on that
 * axis is below min + max, else right, keeping the input order within each
 * side.  Leaves are numbered by the position at which the recursion (left
 * before right) meets them: perm[p] = input index of the leaf at position p.
 * Internal nodes are numbered as in orc_radix_tree (root 0; a child covering
 * positions [lo, split] is numbered split, one covering [split + 1, hi] is
 * split + 1), children c >= 0 internal, c < 0 leaf at position ~c; bb and rep
 * (the leftmost member: min X, then min Y) are given in positions too.  So
 * after reordering the nodes by perm the WSPD code runs on this tree as it
 * does on the radix tree.  Needs N >= 2 and distinct points. */
void orc_split_tree(int64_t N, const int32_t* X, const int32_t* Y, int32_t* perm, int32_t* left,
                    int32_t* right, int32_t* bb, int32_t* rep) {
    if (N < 2) return;
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * N);
    int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * N);
    for (int64_t i = 0; i < N; i++) idx[i] = (int32_t)i;
    int64_t* stk = (int64_t*)malloc(sizeof(int64_t) * 3 * (N + 1));
    int64_t sp = 0;
    stk[sp++] = 0;
    stk[sp++] = N - 1;
    stk[sp++] = 0;
    while (sp > 0) {
        int64_t w = stk[--sp], hi = stk[--sp], lo = stk[--sp];
        int64_t mnx = X[idx[lo]], mxx = mnx, mny = Y[idx[lo]], mxy = mny;
        int32_t r = idx[lo];
        for (int64_t k = lo; k <= hi; k++) {
            int32_t v = idx[k];
            if (X[v] < mnx) mnx = X[v];
            if (X[v] > mxx) mxx = X[v];
            if (Y[v] < mny) mny = Y[v];
            if (Y[v] > mxy) mxy = Y[v];
            if (X[v] < X[r] || (X[v] == X[r] && Y[v] < Y[r])) r = v;
        }
        int by_x = (mxx - mnx) >= (mxy - mny);
        int64_t mid2 = by_x ? mnx + mxx : mny + mxy;
        int64_t nl = 0, nr = 0;
        for (int64_t k = lo; k <= hi; k++) { /* stable partition */
            int32_t v = idx[k];
            int64_t c2 = 2 * (int64_t)(by_x ? X[v] : Y[v]);
            if (c2 < mid2) idx[lo + nl++] = v;
            else tmp[nr++] = v;
        }
        for (int64_t k = 0; k < nr; k++) idx[lo + nl + k] = tmp[k];
        int64_t split = lo + nl - 1; /* both sides are non-empty: min goes left, max right */
        left[w] = (split == lo) ? (int32_t)~lo : (int32_t)split;
        right[w] = (split + 1 == hi) ? (int32_t)~hi : (int32_t)(split + 1);
        bb[4 * w + 0] = (int32_t)mnx;
        bb[4 * w + 1] = (int32_t)mxx;
        bb[4 * w + 2] = (int32_t)mny;
        bb[4 * w + 3] = (int32_t)mxy;
        rep[w] = r; /* an input index for now; positions below */
        if (split != lo) {
            stk[sp++] = lo;
            stk[sp++] = split;
            stk[sp++] = split;
        }
        if (split + 1 != hi) {
            stk[sp++] = split + 1;
            stk[sp++] = hi;
            stk[sp++] = split + 1;
        }
    }
    for (int64_t p = 0; p < N; p++) {
        perm[p] = idx[p];
        pos[idx[p]] = (int32_t)p;
    }
    for (int64_t w = 0; w < N - 1; w++) rep[w] = pos[rep[w]];
    free(idx);
    free(tmp);
    free(pos);
    free(stk);
}

/* ------------------------------------------------------------------------- */
/* s-WSPD (well-separated pairs) and its biarcs.                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t mnx, mxx, mny, mxy;
    int32_t rep;
    int32_t l, r; /* children (internal only) */
    int leaf;
} tnode_t;

typedef struct {
    const int32_t *X, *Y, *left, *right, *bb, *rep;
} tree_t;

static tnode_t get_node(const tree_t* t, int32_t c) {
    tnode_t n;
    if (c < 0) {
        int32_t i = ~c;
        n.mnx = n.mxx = t->X[i];
        n.mny = n.mxy = t->Y[i];
        n.rep = i;
        n.l = n.r = 0;
        n.leaf = 1;
    } else {
        n.mnx = t->bb[4 * c + 0];
        n.mxx = t->bb[4 * c + 1];
        n.mny = t->bb[4 * c + 2];
        n.mxy = t->bb[4 * c + 3];
        n.rep = t->rep[c];
        n.l = t->left[c];
        n.r = t->right[c];
        n.leaf = 0;
    }
    return n;
}

static int64_t max_len(const tnode_t* a) {
    int64_t wx = a->mxx - a->mnx, wy = a->mxy - a->mny;
    return wx > wy ? wx : wy;
}

/* s-well-separated: the two point sets fit in balls of a common radius d
 * whose distance is at least s*d.  With the circumscribed circles of the
 * tight bounding boxes, d = max of the two radii, and in doubled coordinates
 * (centre C = (minX+maxX, minY+maxY), diameter D = bbox diagonal) the test is
 * |C_u - C_v| >= (s+2) max(D_u, D_v), compared squared in 128-bit integers. */
int orc_well_separated(int64_t amnx, int64_t amxx, int64_t amny, int64_t amxy,
                       int64_t bmnx, int64_t bmxx, int64_t bmny, int64_t bmxy, int64_t s) {
    int64_t dx = (amnx + amxx) - (bmnx + bmxx);
    int64_t dy = (amny + amxy) - (bmny + bmxy);
    u128 D2 = (u128)((__int128)dx * dx) + (u128)((__int128)dy * dy);
    int64_t awx = amxx - amnx, awy = amxy - amny, bwx = bmxx - bmnx, bwy = bmxy - bmny;
    u128 ra = (u128)((__int128)awx * awx) + (u128)((__int128)awy * awy);
    u128 rb = (u128)((__int128)bwx * bwx) + (u128)((__int128)bwy * bwy);
    u128 R2 = ra > rb ? ra : rb;
    u128 k = (u128)(s + 2) * (u128)(s + 2);
    return D2 >= k * R2;
}

static int ws_nodes(const tnode_t* a, const tnode_t* b, int64_t s) {
    return orc_well_separated(a->mnx, a->mxx, a->mny, a->mxy, b->mnx, b->mxx, b->mny, b->mxy, s);
}

/* For every internal node w, collect the well-separated pairs below its two
 * children (Algorithms 6-8, run sequentially): a pair that is well separated
 * is emitted as the biarc rep(u)->rep(v), rep(v)->rep(u); otherwise the node
 * with the larger bounding-box side is split (ties split v).  Writes at most
 * cap arcs; returns the total number of directed arcs. */
int64_t orc_wspd(int64_t N, const int32_t* X, const int32_t* Y, const int32_t* left,
                 const int32_t* right, const int32_t* bb, const int32_t* rep, int64_t s,
                 int32_t* tails, int32_t* heads, int64_t cap) {
    if (N < 2) return 0;
    tree_t t = {X, Y, left, right, bb, rep};
    int64_t scap = 1024;
    int32_t* stk = (int32_t*)malloc(sizeof(int32_t) * 2 * scap);
    int64_t m = 0;
    for (int64_t w = 0; w < N - 1; w++) {
        int64_t sp = 0;
        stk[sp++] = left[w];
        stk[sp++] = right[w];
        while (sp > 0) {
            int32_t vb = stk[--sp], ua = stk[--sp];
            tnode_t u = get_node(&t, ua), v = get_node(&t, vb);
            if (ws_nodes(&u, &v, s)) {
                if (m + 2 <= cap) {
                    tails[m] = u.rep;
                    heads[m] = v.rep;
                    tails[m + 1] = v.rep;
                    heads[m + 1] = u.rep;
                }
                m += 2;
                continue;
            }
            if (sp + 4 > 2 * scap) {
                scap *= 2;
                stk = (int32_t*)realloc(stk, sizeof(int32_t) * 2 * scap);
            }
            if (max_len(&u) > max_len(&v)) {
                stk[sp++] = u.r;
                stk[sp++] = vb;
                stk[sp++] = u.l;
                stk[sp++] = vb;
            } else {
                stk[sp++] = ua;
                stk[sp++] = v.r;
                stk[sp++] = ua;
                stk[sp++] = v.l;
            }
        }
    }
    free(stk);
    return m;
}

/* The well-separated pairs themselves (node references as in the tree:
 * c >= 0 internal, c < 0 leaf ~c), in the order orc_wspd visits them.  Used
 * by the pins that check the decomposition against its definition. */
int64_t orc_wspd_pairs(int64_t N, const int32_t* X, const int32_t* Y, const int32_t* left,
                       const int32_t* right, const int32_t* bb, const int32_t* rep, int64_t s,
                       int32_t* pu, int32_t* pv, int64_t cap) {
    if (N < 2) return 0;
    tree_t t = {X, Y, left, right, bb, rep};
    int64_t scap = 1024, m = 0;
    int32_t* stk = (int32_t*)malloc(sizeof(int32_t) * 2 * scap);
    for (int64_t w = 0; w < N - 1; w++) {
        int64_t sp = 0;
        stk[sp++] = left[w];
        stk[sp++] = right[w];
        while (sp > 0) {
            int32_t vb = stk[--sp], ua = stk[--sp];
            tnode_t u = get_node(&t, ua), v = get_node(&t, vb);
            if (ws_nodes(&u, &v, s)) {
                if (m < cap) {
                    pu[m] = ua;
                    pv[m] = vb;
                }
                m++;
                continue;
            }
            if (sp + 4 > 2 * scap) {
                scap *= 2;
                stk = (int32_t*)realloc(stk, sizeof(int32_t) * 2 * scap);
            }
            if (max_len(&u) > max_len(&v)) {
                stk[sp++] = u.r;
                stk[sp++] = vb;
                stk[sp++] = u.l;
                stk[sp++] = vb;
            } else {
                stk[sp++] = ua;
                stk[sp++] = v.r;
                stk[sp++] = ua;
                stk[sp++] = v.l;
            }
        }
    }
    free(stk);
    return m;
}

/* ------------------------------------------------------------------------- */
/* Sparse transshipment network: diagonal arcs + CSR.                        */
/* ------------------------------------------------------------------------- */

/* Node ids: 0..N-1 the condensed nodes (Morton rank), N = ā, N+1 = b̄.
 * Arcs: the WSPD biarcs (cost = rounded-up l2), u->ā for every node holding A
 * mass and b̄->v for every node holding B mass (cost = rounded-up distance to
 * the diagonal, Algorithm 9), and b̄->ā at cost 0 (the zero-weight edges
 * between the two sets of diagonal projections in Bi(A,B)).  Arcs are sorted
 * by (tail, head); row_ptr has N+3 entries.  Supplies: sigma(u) = cntA - cntB,
 * sigma(ā) = -F_A, sigma(b̄) = F_B.  Returns the number of arcs m. */
int64_t orc_build_network(int64_t N, const int32_t* X, const int32_t* Y, const int64_t* cntA,
                          const int64_t* cntB, int64_t nws, const int32_t* wt, const int32_t* wh,
                          int64_t* row_ptr, int32_t* head, int64_t* cost, int64_t* supply, int64_t kappa, int64_t tau) {
    int64_t na = 0, nb = 0, FA = 0, FB = 0;
    for (int64_t i = 0; i < N; i++) {
        if (cntA[i] > 0) na++;
        if (cntB[i] > 0) nb++;
        FA += cntA[i];
        FB += cntB[i];
    }
    int64_t m = nws + na + nb + 1;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * m);
    int64_t k = 0;
    for (int64_t i = 0; i < nws; i++) key[k++] = ((uint64_t)wt[i] << 32) | (uint32_t)wh[i];
    for (int64_t i = 0; i < N; i++) {
        if (cntA[i] > 0) key[k++] = ((uint64_t)i << 32) | (uint64_t)N;
        if (cntB[i] > 0) key[k++] = ((uint64_t)(N + 1) << 32) | (uint64_t)i;
    }
    key[k++] = ((uint64_t)(N + 1) << 32) | (uint64_t)N;
    qsort(key, m, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 0; i <= N + 2; i++) row_ptr[i] = 0;
    for (int64_t a = 0; a < m; a++) {
        int64_t u = (int64_t)(key[a] >> 32), v = (int64_t)(key[a] & 0xffffffffu);
        row_ptr[u + 1]++;
        head[a] = (int32_t)v;
        if (u < N && v < N)
            cost[a] = orc_cost(X[u], Y[u], X[v], Y[v]);
        else if (u < N && v == N)
            cost[a] = orc_cmake(X[u], Y[u], kappa, tau);
        else if (u == N + 1 && v < N)
            cost[a] = orc_cmake(X[v], Y[v], kappa, tau);
        else
            cost[a] = 0;
    }
    for (int64_t i = 0; i < N + 2; i++) row_ptr[i + 1] += row_ptr[i];
    for (int64_t i = 0; i < N; i++) supply[i] = cntA[i] - cntB[i];
    supply[N] = -FA;
    supply[N + 1] = FB;
    free(key);
    return m;
}

/* ------------------------------------------------------------------------- */
/* Network simplex with block search pivoting (run to optimality).           */
/* Two instantiations: exact int64 costs, and double costs for exact W1.     */
/* ------------------------------------------------------------------------- */

#define NS_COST int64_t
#define NS_FN(x) x##_int
#define NS_ELIGIBLE(rc, tol) ((rc) < 0)
#include "netsimplex.inc"
#undef NS_COST
#undef NS_FN
#undef NS_ELIGIBLE

#define NS_COST double
#define NS_FN(x) x##_dbl
#define NS_ELIGIBLE(rc, tol) ((rc) < -(tol))
#include "netsimplex.inc"
#undef NS_COST
#undef NS_FN
#undef NS_ELIGIBLE

/* Solve the min-cost flow on a CSR network.  Returns 0 on success, 1 if
 * infeasible, 2 if the pivot cap was reached.  *opt is the optimum (int64). */
int orc_mcf_csr(int64_t n, const int64_t* row_ptr, const int32_t* head, const int64_t* cost,
                const int64_t* supply, int64_t* flow, int64_t* pot, int64_t* opt,
                int64_t* pivots, int64_t max_pivots) {
    int64_t m = row_ptr[n];
    int32_t* tail = (int32_t*)malloc(sizeof(int32_t) * (m > 0 ? m : 1));
    for (int64_t u = 0; u < n; u++)
        for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; a++) tail[a] = (int32_t)u;
    int st = ns_solve_int(n, m, tail, head, cost, supply, flow, pot, opt, pivots, max_pivots, 0.0);
    free(tail);
    return st;
}

/* Same on an arc list (tails, heads). */
int orc_mcf_arcs(int64_t n, int64_t m, const int32_t* tail, const int32_t* head,
                 const int64_t* cost, const int64_t* supply, int64_t* flow, int64_t* pot,
                 int64_t* opt, int64_t* pivots, int64_t max_pivots) {
    return ns_solve_int(n, m, tail, head, cost, supply, flow, pot, opt, pivots, max_pivots, 0.0);
}

int orc_mcf_arcs_dbl(int64_t n, int64_t m, const int32_t* tail, const int32_t* head,
                     const double* cost, const int64_t* supply, int64_t* flow, double* pot,
                     double* opt, int64_t* pivots, int64_t max_pivots, double tol) {
    return ns_solve_dbl(n, m, tail, head, cost, supply, flow, pot, opt, pivots, max_pivots, tol);
}

/* ------------------------------------------------------------------------- */
/* Dense networks G(A,B) for the invariants and for the exact W1.            */
/* ------------------------------------------------------------------------- */

/* Integer optimum of the dense bipartite network G(A,B) on weighted node sets
 * P (A side) and Q (B side) with rounded-up costs: arcs P x Q, P -> ā,
 * b̄ -> Q, b̄ -> ā.  Coincident nodes of P and Q stay separate (cost 0). */
int orc_dense_opt_int(const int32_t* PX, const int32_t* PY, const int64_t* Pc, int64_t nP,
                      const int32_t* QX, const int32_t* QY, const int64_t* Qc, int64_t nQ,
                      int64_t kappa, int64_t tau, int64_t* opt, int64_t max_pivots) {
    int64_t n = nP + nQ + 2, abar = nP + nQ, bbar = nP + nQ + 1;
    int64_t m = nP * nQ + nP + nQ + 1;
    int32_t* t = (int32_t*)malloc(sizeof(int32_t) * m);
    int32_t* h = (int32_t*)malloc(sizeof(int32_t) * m);
    int64_t* c = (int64_t*)malloc(sizeof(int64_t) * m);
    int64_t* sup = (int64_t*)malloc(sizeof(int64_t) * n);
    int64_t* f = (int64_t*)malloc(sizeof(int64_t) * m);
    int64_t* pot = (int64_t*)malloc(sizeof(int64_t) * n);
    int64_t k = 0, FA = 0, FB = 0;
    for (int64_t u = 0; u < nP; u++)
        for (int64_t v = 0; v < nQ; v++) {
            t[k] = (int32_t)u;
            h[k] = (int32_t)(nP + v);
            c[k] = orc_cost(PX[u], PY[u], QX[v], QY[v]);
            k++;
        }
    for (int64_t u = 0; u < nP; u++) {
        t[k] = (int32_t)u;
        h[k] = (int32_t)abar;
        c[k] = orc_cmake(PX[u], PY[u], kappa, tau);
        k++;
        sup[u] = Pc[u];
        FA += Pc[u];
    }
    for (int64_t v = 0; v < nQ; v++) {
        t[k] = (int32_t)bbar;
        h[k] = (int32_t)(nP + v);
        c[k] = orc_cmake(QX[v], QY[v], kappa, tau);
        k++;
        sup[nP + v] = -Qc[v];
        FB += Qc[v];
    }
    t[k] = (int32_t)bbar;
    h[k] = (int32_t)abar;
    c[k] = 0;
    k++;
    sup[abar] = -FA;
    sup[bbar] = FB;
    int64_t piv;
    int st = ns_solve_int(n, m, t, h, c, sup, f, pot, opt, &piv, max_pivots, 0.0);
    free(t);
    free(h);
    free(c);
    free(sup);
    free(f);
    free(pot);
    return st;
}

typedef struct {
    double b, d;
} dpt_t;

static int cmp_dpt(const void* a, const void* b) {
    const dpt_t* p = (const dpt_t*)a;
    const dpt_t* q = (const dpt_t*)b;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->d != q->d) return p->d < q->d ? -1 : 1;
    return 0;
}

static int64_t condense_dbl(const double* bd, int64_t n, double* ob, double* od, int64_t* oc) {
    dpt_t* p = (dpt_t*)malloc(sizeof(dpt_t) * (n > 0 ? n : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {
        if (bd[2 * i] == bd[2 * i + 1]) continue;
        p[k].b = bd[2 * i];
        p[k].d = bd[2 * i + 1];
        k++;
    }
    qsort(p, k, sizeof(dpt_t), cmp_dpt);
    int64_t m = 0;
    for (int64_t i = 0; i < k; i++) {
        if (i == 0 || cmp_dpt(&p[i], &p[i - 1]) != 0) {
            ob[m] = p[i].b;
            od[m] = p[i].d;
            oc[m] = 0;
            m++;
        }
        oc[m - 1]++;
    }
    free(p);
    return m;
}

/* Exact W1 (Problem 1) with the l2 ground metric, in FP64, on unquantised
 * diagrams given as interleaved (b, d) doubles: min-cost flow on the dense
 * 0-condensed network G(A,B), which by Proposition (matching iff flow) equals
 * the optimal partial matching.  Diagonal arcs cost kappa * d_diag + tau (1
 * and 0 for persistence diagrams; the Conclusion's unbalanced transport
 * otherwise).  Returns W1, or -1 on failure. */
double orc_w1_exact(const double* A, int64_t nA, const double* B, int64_t nB, double kappa, double tau,
                    int64_t max_pivots) {
    double* ab = (double*)malloc(sizeof(double) * (nA + 1));
    double* ad = (double*)malloc(sizeof(double) * (nA + 1));
    int64_t* ac = (int64_t*)malloc(sizeof(int64_t) * (nA + 1));
    double* bb = (double*)malloc(sizeof(double) * (nB + 1));
    double* bdd = (double*)malloc(sizeof(double) * (nB + 1));
    int64_t* bc = (int64_t*)malloc(sizeof(int64_t) * (nB + 1));
    int64_t na = condense_dbl(A, nA, ab, ad, ac);
    int64_t nb = condense_dbl(B, nB, bb, bdd, bc);
    int64_t n = na + nb + 2, abar = na + nb, bbar = na + nb + 1;
    int64_t m = na * nb + na + nb + 1;
    int32_t* t = (int32_t*)malloc(sizeof(int32_t) * m);
    int32_t* h = (int32_t*)malloc(sizeof(int32_t) * m);
    double* c = (double*)malloc(sizeof(double) * m);
    int64_t* sup = (int64_t*)malloc(sizeof(int64_t) * n);
    int64_t* f = (int64_t*)malloc(sizeof(int64_t) * m);
    double* pot = (double*)malloc(sizeof(double) * n);
    int64_t k = 0, FA = 0, FB = 0;
    double cmax = 0.0;
    for (int64_t u = 0; u < na; u++)
        for (int64_t v = 0; v < nb; v++) {
            t[k] = (int32_t)u;
            h[k] = (int32_t)(na + v);
            c[k] = hypot(ab[u] - bb[v], ad[u] - bdd[v]);
            if (c[k] > cmax) cmax = c[k];
            k++;
        }
    for (int64_t u = 0; u < na; u++) {
        t[k] = (int32_t)u;
        h[k] = (int32_t)abar;
        c[k] = kappa * fabs(ad[u] - ab[u]) / sqrt(2.0) + tau;
        if (c[k] > cmax) cmax = c[k];
        k++;
        sup[u] = ac[u];
        FA += ac[u];
    }
    for (int64_t v = 0; v < nb; v++) {
        t[k] = (int32_t)bbar;
        h[k] = (int32_t)(na + v);
        c[k] = kappa * fabs(bdd[v] - bb[v]) / sqrt(2.0) + tau;
        if (c[k] > cmax) cmax = c[k];
        k++;
        sup[na + v] = -bc[v];
        FB += bc[v];
    }
    t[k] = (int32_t)bbar;
    h[k] = (int32_t)abar;
    c[k] = 0.0;
    k++;
    sup[abar] = -FA;
    sup[bbar] = FB;
    double opt = -1.0;
    int64_t piv;
    int st = ns_solve_dbl(n, m, t, h, c, sup, f, pot, &opt, &piv, max_pivots, 1e-12 * (cmax + 1.0));
    if (st != 0) opt = -1.0;
    free(ab);
    free(ad);
    free(ac);
    free(bb);
    free(bdd);
    free(bc);
    free(t);
    free(h);
    free(c);
    free(sup);
    free(f);
    free(pot);
    return opt;
}
