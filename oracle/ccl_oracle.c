/*
 * CPU oracle for two-pass connected-component labelling (PARemSP paper, arXiv 1606.05973).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared object that the
 * tests, the smoke check and the benchmark's CPU-baseline leg load.  The GPU library never
 * links, includes or calls it, and it shares no code with the GPU library.
 *
 * Problem (Section III): label every object pixel (non-zero byte) of a binary image so
 * that 8-connected object pixels share a label.  The result is made unique by numbering:
 * background 0, components 1..K in raster order of their first pixel.
 *
 * What is here, each following the paper's own sequential and parallel algorithms:
 *   oracle_cclremsp  Algorithm 1 (CCLRemSP): Algorithm 4's raster scan with the decision
 *                    tree of Fig. 2, Algorithm 2 (merge, Rem's union with splicing),
 *                    Algorithm 3 (flatten) and the labelling pass.  Its output is already
 *                    in the canonical numbering (see the note before the function).
 *                    With conn = 4 it uses the 4-neighbour mask (b, d) instead.
 *   oracle_aremsp    Algorithm 5 (ARemSP): Algorithm 6's two-rows-at-a-time scan, merge,
 *                    flatten, labelling pass, then a first-occurrence renumbering.
 *   oracle_paremsp   Algorithm 7 (PARemSP) with Algorithm 8 (merger) on OpenMP threads,
 *                    then the same renumbering.
 *   oracle_bfs       breadth-first flood fill straight from the definition (4 or 8).
 *   oracle_bfs_classes  the same flood fill where neighbours connect only when their
 *                    bytes are equal and non-zero (multi-class labelling).
 *
 * Readings taken where the paper's pseudocode is incomplete (each also listed in the
 * design notes):
 *   - Algorithm 6, e=1, d=0, b=0, f=1, a=1: "merge(p,label(a))" lacks an operand; it is
 *     read as merge(p, label(e), label(a)).
 *   - Algorithm 6, e=0, g=1, d=0, f=0: the new label belongs to g (e is background).
 *   - count starts at 1; flatten visits 1..count-1; label 0 with p[0]=0 is background.
 *   - Algorithm 6 with an odd number of rows: the missing second row is background.
 *   - Algorithm 7: each thread's first label is start_row*W + 1 (label 0 is background);
 *     chunks are an even number of rows, the last chunk takes the remainder; rows above a
 *     chunk are background during its local scan; flatten walks each chunk's used label
 *     range in chunk order with one shared k; the labelling pass is parallel.
 *   - Algorithm 8: the locked root link is a compare-and-swap on p[root]; the unlocked
 *     splice is a compare-and-swap from the parent value read, retried when it fails.
 *   - Object pixel = any non-zero byte; pixels outside the image are background.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int32_t lab_t;

#define ORACLE_ERR_ARG (-2)
#define ORACLE_ERR_NOMEM (-1)

/* ---------------------------------------------------------------------------------- */
/* Algorithm 2: merge(p, x, y), Rem's union with splicing.  Keeps p[v] <= v, so the root
 * of every set is its smallest label.  Returns a label of the united set. */
static lab_t rem_merge(lab_t *p, lab_t x, lab_t y)
{
    lab_t rootx = x;
    lab_t rooty = y;
    while (p[rootx] != p[rooty]) {
        if (p[rootx] > p[rooty]) {
            if (rootx == p[rootx]) {
                p[rootx] = p[rooty];
                return p[rootx];
            }
            lab_t z = p[rootx];
            p[rootx] = p[rooty];
            rootx = z;
        } else {
            if (rooty == p[rooty]) {
                p[rooty] = p[rootx];
                return p[rootx];
            }
            lab_t z = p[rooty];
            p[rooty] = p[rootx];
            rooty = z;
        }
    }
    return p[rootx];
}

/* Algorithm 3: flatten(p, count) over provisional labels 1..count-1.  Roots (p[i] == i)
 * receive consecutive final labels k = 1, 2, ... in increasing label order; every other
 * label copies its parent's final label (its parent is smaller, so already final).
 * Returns the number of components. */
static lab_t flatten_labels(lab_t *p, lab_t count)
{
    lab_t k = 1;
    for (lab_t i = 1; i < count; i++) {
        if (p[i] < i) {
            p[i] = p[p[i]];
        } else {
            p[i] = k;
            k++;
        }
    }
    return k - 1;
}

typedef struct {
    const uint8_t *img;
    int64_t h, w, pitch;
    int64_t r0, r1; /* rows [r0, r1) are visible; everything else is background */
} view_t;

static inline int fg(const view_t *v, int64_t y, int64_t x)
{
    if (y < v->r0 || y >= v->r1 || x < 0 || x >= v->w)
        return 0;
    return v->img[y * v->pitch + x] != 0;
}

#define LAB(y, x) label[(y) * w + (x)]

/* ---------------------------------------------------------------------------------- */
/* Algorithm 4 (Scan_CCLRemSP) with the decision tree of Fig. 2.  Mask (Fig. 1a):
 *     a b c
 *     d e
 * copy(x) sets label(e) = p[label(x)]; copy(x, y) sets label(e) = merge(p, label(x),
 * label(y)); new label sets label(e) = count, p[count] = count, count++. */
static lab_t scan_cclremsp8(const view_t *v, lab_t *label, lab_t *p)
{
    const int64_t h = v->h, w = v->w;
    lab_t count = 1;
    p[0] = 0;
    for (int64_t y = 0; y < h; y++) {
        for (int64_t x = 0; x < w; x++) {
            if (!fg(v, y, x)) {
                LAB(y, x) = 0;
                continue;
            }
            if (fg(v, y - 1, x)) {
                LAB(y, x) = p[LAB(y - 1, x)];                                  /* copy(b) */
            } else if (fg(v, y - 1, x + 1)) {
                if (fg(v, y - 1, x - 1)) {
                    LAB(y, x) = rem_merge(p, LAB(y - 1, x + 1), LAB(y - 1, x - 1)); /* copy(c,a) */
                } else if (fg(v, y, x - 1)) {
                    LAB(y, x) = rem_merge(p, LAB(y - 1, x + 1), LAB(y, x - 1));     /* copy(c,d) */
                } else {
                    LAB(y, x) = p[LAB(y - 1, x + 1)];                          /* copy(c) */
                }
            } else if (fg(v, y - 1, x - 1)) {
                LAB(y, x) = p[LAB(y - 1, x - 1)];                              /* copy(a) */
            } else if (fg(v, y, x - 1)) {
                LAB(y, x) = p[LAB(y, x - 1)];                                  /* copy(d) */
            } else {
                LAB(y, x) = count;                                             /* new label */
                p[count] = count;
                count++;
            }
        }
    }
    return count;
}

/* The paper names 4-connectivity but uses only 8 (Section III).  The 4-neighbour scan
 * keeps the same structure with the mask reduced to b (above) and d (left). */
static lab_t scan_cclremsp4(const view_t *v, lab_t *label, lab_t *p)
{
    const int64_t h = v->h, w = v->w;
    lab_t count = 1;
    p[0] = 0;
    for (int64_t y = 0; y < h; y++) {
        for (int64_t x = 0; x < w; x++) {
            if (!fg(v, y, x)) {
                LAB(y, x) = 0;
                continue;
            }
            if (fg(v, y - 1, x)) {
                if (fg(v, y, x - 1)) {
                    LAB(y, x) = rem_merge(p, LAB(y - 1, x), LAB(y, x - 1));   /* copy(b,d) */
                } else {
                    LAB(y, x) = p[LAB(y - 1, x)];                              /* copy(b) */
                }
            } else if (fg(v, y, x - 1)) {
                LAB(y, x) = p[LAB(y, x - 1)];                                  /* copy(d) */
            } else {
                LAB(y, x) = count;                                             /* new label */
                p[count] = count;
                count++;
            }
        }
    }
    return count;
}

/* Why CCLRemSP's output is canonical without renumbering: the raster-first pixel of a
 * component has no earlier object neighbour, so it takes a new label, and that label is
 * the smallest one its component ever holds; Rem's merge keeps p[v] <= v, so the root of
 * each set is that label; flatten numbers roots in increasing order, i.e. in raster order
 * of first pixels. */
int64_t oracle_cclremsp(const uint8_t *img, int64_t h, int64_t w, int64_t pitch, int32_t conn,
                        int32_t *label)
{
    if (h < 0 || w < 0 || (h > 0 && w > 0 && (!img || !label || pitch < w)))
        return ORACLE_ERR_ARG;
    if (conn != 4 && conn != 8)
        return ORACLE_ERR_ARG;
    if (h == 0 || w == 0)
        return 0;
    /* new labels in one row are never adjacent, so at most ceil(W/2) per row */
    size_t cap = (size_t)h * (size_t)((w + 1) / 2) + 2;
    lab_t *p = (lab_t *)malloc(cap * sizeof(lab_t));
    if (!p)
        return ORACLE_ERR_NOMEM;
    view_t v = {img, h, w, pitch, 0, h};
    lab_t count = (conn == 8) ? scan_cclremsp8(&v, label, p) : scan_cclremsp4(&v, label, p);
    lab_t k = flatten_labels(p, count);
    for (int64_t y = 0; y < h; y++)                 /* labelling pass (Algorithm 1) */
        for (int64_t x = 0; x < w; x++)
            LAB(y, x) = p[LAB(y, x)];
    free(p);
    return k;
}

/* ---------------------------------------------------------------------------------- */
/* Algorithm 6 (Scan_ARemSP): rows [v->r0, v->r1) in pairs (e row i, g row i+1), one column
 * at a time.  Mask (Fig. 1b):
 *     a b c        row i-1
 *     d e          row i
 *     f g          row i+1
 * Labels start at *count (updated).  Background pixels of the scanned rows get 0. */
static void scan_aremsp(const view_t *v, lab_t *label, lab_t *p, lab_t *count)
{
    const int64_t w = v->w;
    lab_t cnt = *count;
    for (int64_t i = v->r0; i < v->r1; i += 2) {
        const int has_g = (i + 1 < v->r1);
        for (int64_t x = 0; x < w; x++) {
            const int e = fg(v, i, x);
            const int g = fg(v, i + 1, x);
            const int a = fg(v, i - 1, x - 1);
            const int b = fg(v, i - 1, x);
            const int c = fg(v, i - 1, x + 1);
            const int d = fg(v, i, x - 1);
            const int f = fg(v, i + 1, x - 1);
            if (e) {
                if (!d) {
                    if (b) {
                        LAB(i, x) = LAB(i - 1, x);
                        if (f)
                            rem_merge(p, LAB(i, x), LAB(i + 1, x - 1));
                    } else {
                        if (f) {
                            LAB(i, x) = LAB(i + 1, x - 1);
                            if (a)
                                rem_merge(p, LAB(i, x), LAB(i - 1, x - 1));
                            if (c)
                                rem_merge(p, LAB(i, x), LAB(i - 1, x + 1));
                        } else {
                            if (a) {
                                LAB(i, x) = LAB(i - 1, x - 1);
                                if (c)
                                    rem_merge(p, LAB(i, x), LAB(i - 1, x + 1));
                            } else {
                                if (c) {
                                    LAB(i, x) = LAB(i - 1, x + 1);
                                } else {
                                    LAB(i, x) = cnt;
                                    p[cnt] = cnt;
                                    cnt++;
                                }
                            }
                        }
                    }
                } else {
                    LAB(i, x) = LAB(i, x - 1);
                    if (!b) {
                        if (c)
                            rem_merge(p, LAB(i, x), LAB(i - 1, x + 1));
                    }
                }
                if (g)
                    LAB(i + 1, x) = LAB(i, x);
                else if (has_g)
                    LAB(i + 1, x) = 0;
            } else {
                LAB(i, x) = 0;
                if (g) {
                    if (d) {
                        LAB(i + 1, x) = LAB(i, x - 1);
                    } else {
                        if (f) {
                            LAB(i + 1, x) = LAB(i + 1, x - 1);
                        } else {
                            LAB(i + 1, x) = cnt;
                            p[cnt] = cnt;
                            cnt++;
                        }
                    }
                } else if (has_g) {
                    LAB(i + 1, x) = 0;
                }
            }
        }
    }
    *count = cnt;
}

/* Renumber labels 1..K by first occurrence in raster order (the canonical numbering).
 * The paper's flatten numbers components by smallest provisional label, which for the
 * two-row scan is column-pair order, not raster order. */
int64_t oracle_canonicalize(int32_t *label, int64_t n, int64_t k)
{
    if (n < 0 || k < 0 || (n > 0 && !label))
        return ORACLE_ERR_ARG;
    lab_t *map = (lab_t *)calloc((size_t)k + 1, sizeof(lab_t));
    if (!map)
        return ORACLE_ERR_NOMEM;
    lab_t next = 1;
    for (int64_t i = 0; i < n; i++) {
        lab_t l = label[i];
        if (l == 0)
            continue;
        if (l < 0 || l > k) {
            free(map);
            return ORACLE_ERR_ARG;
        }
        if (map[l] == 0)
            map[l] = next++;
        label[i] = map[l];
    }
    free(map);
    return next - 1;
}

/* Algorithm 5 (ARemSP): scan, flatten, labelling pass; renumbered when remap != 0. */
int64_t oracle_aremsp(const uint8_t *img, int64_t h, int64_t w, int64_t pitch, int32_t *label,
                      int32_t remap)
{
    if (h < 0 || w < 0 || (h > 0 && w > 0 && (!img || !label || pitch < w)))
        return ORACLE_ERR_ARG;
    if (h == 0 || w == 0)
        return 0;
    /* at most one new label per column pair, never in adjacent columns */
    size_t cap = (size_t)((h + 1) / 2) * (size_t)((w + 1) / 2) + 2;
    lab_t *p = (lab_t *)malloc(cap * sizeof(lab_t));
    if (!p)
        return ORACLE_ERR_NOMEM;
    view_t v = {img, h, w, pitch, 0, h};
    lab_t count = 1;
    p[0] = 0;
    scan_aremsp(&v, label, p, &count);
    lab_t k = flatten_labels(p, count);
    for (int64_t y = 0; y < h; y++)
        for (int64_t x = 0; x < w; x++)
            LAB(y, x) = p[LAB(y, x)];
    free(p);
    if (remap)
        return oracle_canonicalize(label, h * w, k);
    return k;
}

/* ---------------------------------------------------------------------------------- */
/* Algorithm 8 (merger): Rem's union for concurrent threads.  The paper takes a lock on the
 * root, re-checks that it is still a root and links it; here that is one compare-and-swap
 * of p[root] from root to the other parent.  The paper's splice p[rootx] <- p[rooty] is an
 * unlocked write; here it too is a compare-and-swap from the parent value this thread read
 * (a failed one re-reads and retries).  An unconditional splice can overwrite a parent that
 * another thread has just set, detaching a subtree that no thread then reconnects. */
static inline lab_t ld(lab_t *p, lab_t i) { return __atomic_load_n(&p[i], __ATOMIC_ACQUIRE); }

static inline int cas_lab(lab_t *addr, lab_t expect, lab_t val)
{
    return __atomic_compare_exchange_n(addr, &expect, val, 0, __ATOMIC_ACQ_REL, __ATOMIC_ACQUIRE);
}

static void rem_merger(lab_t *p, lab_t x, lab_t y)
{
    lab_t rootx = x;
    lab_t rooty = y;
    for (;;) {
        lab_t px = ld(p, rootx);
        lab_t py = ld(p, rooty);
        if (px == py)
            return;
        if (px > py) {
            if (!cas_lab(&p[rootx], px, py))
                continue; /* p[rootx] changed since it was read: read again */
            if (rootx == px)
                return; /* a root was linked */
            rootx = px;
        } else {
            if (!cas_lab(&p[rooty], py, px))
                continue;
            if (rooty == py)
                return;
            rooty = py;
        }
    }
}

/* Algorithm 7 (PARemSP).  Threads take chunks of an even number of rows; each runs
 * Scan_ARemSP on its chunk with its own label range starting at start_row*W + 1; then the
 * first row of every chunk but the first is merged with the row above it using the same
 * decision as the paper's boundary loop (b, else a and c); then flatten and labelling. */
int64_t oracle_paremsp(const uint8_t *img, int64_t h, int64_t w, int64_t pitch, int32_t *label,
                       int32_t nthreads, int32_t remap)
{
    if (h < 0 || w < 0 || (h > 0 && w > 0 && (!img || !label || pitch < w)) || nthreads < 1)
        return ORACLE_ERR_ARG;
    if (h == 0 || w == 0)
        return 0;
    if ((uint64_t)h * (uint64_t)w + 2 > (uint64_t)INT32_MAX)
        return ORACLE_ERR_ARG;
    const int64_t numiter = (h + 1) / 2; /* row pairs */
    int64_t nt = nthreads;
    if (nt > numiter)
        nt = numiter;
    const int64_t chunk = numiter / nt;
    lab_t *p = (lab_t *)malloc(((size_t)h * (size_t)w + 2) * sizeof(lab_t));
    int64_t *start = (int64_t *)malloc((size_t)(nt + 1) * sizeof(int64_t));
    lab_t *cend = (lab_t *)malloc((size_t)nt * sizeof(lab_t));
    if (!p || !start || !cend) {
        free(p);
        free(start);
        free(cend);
        return ORACLE_ERR_NOMEM;
    }
    for (int64_t t = 0; t < nt; t++)
        start[t] = 2 * chunk * t;
    start[nt] = h;
    p[0] = 0;

#pragma omp parallel for num_threads(nt) schedule(static, 1)
    for (int64_t t = 0; t < nt; t++) {
        view_t v = {img, h, w, pitch, start[t], start[t + 1]};
        lab_t count = (lab_t)(start[t] * w + 1);
        scan_aremsp(&v, label, p, &count);
        cend[t] = count;
    }

#pragma omp parallel for num_threads(nt) schedule(static, 1)
    for (int64_t t = 1; t < nt; t++) {
        const int64_t i = start[t];
        for (int64_t x = 0; x < w; x++) {
            lab_t e = LAB(i, x);
            if (e == 0)
                continue;
            if (LAB(i - 1, x) != 0) {
                rem_merger(p, e, LAB(i - 1, x));
            } else {
                if (x > 0 && LAB(i - 1, x - 1) != 0)
                    rem_merger(p, e, LAB(i - 1, x - 1));
                if (x + 1 < w && LAB(i - 1, x + 1) != 0)
                    rem_merger(p, e, LAB(i - 1, x + 1));
            }
        }
    }

    /* flatten over each chunk's used label range, in chunk order, with one shared k */
    lab_t k = 1;
    for (int64_t t = 0; t < nt; t++) {
        for (lab_t i = (lab_t)(start[t] * w + 1); i < cend[t]; i++) {
            if (p[i] < i) {
                p[i] = p[p[i]];
            } else {
                p[i] = k;
                k++;
            }
        }
    }

#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t y = 0; y < h; y++)
        for (int64_t x = 0; x < w; x++)
            LAB(y, x) = p[LAB(y, x)];

    free(p);
    free(start);
    free(cend);
    if (remap)
        return oracle_canonicalize(label, h * w, k - 1);
    return k - 1;
}

/* ---------------------------------------------------------------------------------- */
/* Flood fill straight from the definition: scanning in raster order, every unlabelled
 * object pixel opens a new component that a breadth-first search spreads over its 4- or
 * 8-neighbours.  Numbering is canonical by construction. */
int64_t oracle_bfs(const uint8_t *img, int64_t h, int64_t w, int64_t pitch, int32_t conn,
                   int32_t *label)
{
    if (h < 0 || w < 0 || (h > 0 && w > 0 && (!img || !label || pitch < w)))
        return ORACLE_ERR_ARG;
    if (conn != 4 && conn != 8)
        return ORACLE_ERR_ARG;
    if (h == 0 || w == 0)
        return 0;
    int64_t n = h * w;
    int64_t *queue = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!queue)
        return ORACLE_ERR_NOMEM;
    memset(label, 0, (size_t)n * sizeof(int32_t));
    static const int dy8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    static const int dx8[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    static const int dy4[4] = {-1, 0, 0, 1};
    static const int dx4[4] = {0, -1, 1, 0};
    const int *dy = conn == 8 ? dy8 : dy4;
    const int *dx = conn == 8 ? dx8 : dx4;
    lab_t k = 0;
    for (int64_t s = 0; s < n; s++) {
        int64_t sy = s / w, sx = s % w;
        if (img[sy * pitch + sx] == 0 || label[s] != 0)
            continue;
        k++;
        int64_t qh = 0, qt = 0;
        queue[qt++] = s;
        label[s] = k;
        while (qh < qt) {
            int64_t q = queue[qh++];
            int64_t qy = q / w, qx = q % w;
            for (int j = 0; j < conn; j++) {
                int64_t ny = qy + dy[j], nx = qx + dx[j];
                if (ny < 0 || ny >= h || nx < 0 || nx >= w)
                    continue;
                if (img[ny * pitch + nx] == 0 || label[ny * w + nx] != 0)
                    continue;
                label[ny * w + nx] = k;
                queue[qt++] = ny * w + nx;
            }
        }
    }
    free(queue);
    return k;
}

/* Multi-class labelling, from the definition: two pixels are connected when they are
 * 4- or 8-neighbours with the same non-zero value (a class, e.g. a land-cover code; the
 * paper's Section V labels binarised rasters and notes the method extends to such data).
 * Breadth-first flood fill in raster order, so the numbering is canonical. */
int64_t oracle_bfs_classes(const uint8_t *img, int64_t h, int64_t w, int64_t pitch, int32_t conn,
                           int32_t *label)
{
    if (h < 0 || w < 0 || (h > 0 && w > 0 && (!img || !label || pitch < w)))
        return ORACLE_ERR_ARG;
    if (conn != 4 && conn != 8)
        return ORACLE_ERR_ARG;
    if (h == 0 || w == 0)
        return 0;
    int64_t n = h * w;
    int64_t *queue = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!queue)
        return ORACLE_ERR_NOMEM;
    memset(label, 0, (size_t)n * sizeof(int32_t));
    static const int dy8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    static const int dx8[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    static const int dy4[4] = {-1, 0, 0, 1};
    static const int dx4[4] = {0, -1, 1, 0};
    const int *dy = conn == 8 ? dy8 : dy4;
    const int *dx = conn == 8 ? dx8 : dx4;
    lab_t k = 0;
    for (int64_t s = 0; s < n; s++) {
        int64_t sy = s / w, sx = s % w;
        const uint8_t cls = img[sy * pitch + sx];
        if (cls == 0 || label[s] != 0)
            continue;
        k++;
        int64_t qh = 0, qt = 0;
        queue[qt++] = s;
        label[s] = k;
        while (qh < qt) {
            int64_t q = queue[qh++];
            int64_t qy = q / w, qx = q % w;
            for (int j = 0; j < conn; j++) {
                int64_t ny = qy + dy[j], nx = qx + dx[j];
                if (ny < 0 || ny >= h || nx < 0 || nx >= w)
                    continue;
                if (img[ny * pitch + nx] != cls || label[ny * w + nx] != 0)
                    continue;
                label[ny * w + nx] = k;
                queue[qt++] = ny * w + nx;
            }
        }
    }
    free(queue);
    return k;
}

int32_t oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
