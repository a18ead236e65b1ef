/*
 * Input generator helper (not part of the method): 0-dimensional persistence
 * of the lower-star filtration of an 8-bit image, the kind of diagram the
 * paper's image datasets produce.  Pixels enter in increasing value (ties by
 * index); a pixel joins its already-present 4-neighbours; when two components
 * meet, the younger one (later minimum) dies at the current value (elder
 * rule).  The essential class and zero-persistence pairs are not reported.
 */
#include <stdint.h>
#include <stdlib.h>

static int32_t uf_find(int32_t* parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

/* img: H*W uint8, row-major.  out: up to cap (birth, death) uint8 pairs.
 * Returns the number of pairs written. */
int64_t synth_lowerstar_h0(const uint8_t* img, int32_t H, int32_t W, uint8_t* out, int64_t cap) {
    int64_t n = (int64_t)H * W;
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * n);
    int64_t start[257] = {0};
    for (int64_t i = 0; i < n; i++) start[img[i] + 1]++;
    for (int v = 0; v < 256; v++) start[v + 1] += start[v];
    for (int64_t i = 0; i < n; i++) order[start[img[i]]++] = (int32_t)i;
    for (int64_t i = 0; i < n; i++) {
        rank[order[i]] = (int32_t)i;
        parent[i] = -1;
    }
    int64_t m = 0;
    for (int64_t t = 0; t < n; t++) {
        int32_t p = order[t];
        parent[p] = p;
        int32_t y = p / W, x = p % W;
        int32_t nb[4] = {-1, -1, -1, -1};
        if (x > 0) nb[0] = p - 1;
        if (x + 1 < W) nb[1] = p + 1;
        if (y > 0) nb[2] = p - W;
        if (y + 1 < H) nb[3] = p + W;
        for (int k = 0; k < 4; k++) {
            int32_t q = nb[k];
            if (q < 0 || parent[q] < 0) continue;
            int32_t rp = uf_find(parent, p), rq = uf_find(parent, q);
            if (rp == rq) continue;
            /* the root of a component is its oldest pixel (smallest rank) */
            int32_t old = rank[rp] < rank[rq] ? rp : rq;
            int32_t young = old == rp ? rq : rp;
            if (img[young] < img[p] && m < cap) {
                out[2 * m] = img[young];
                out[2 * m + 1] = img[p];
                m++;
            }
            parent[young] = old;
        }
    }
    free(order);
    free(rank);
    free(parent);
    return m;
}
