// Tile-level phases of the GPU labelling path, written once as __host__ __device__
// functions.  The CUDA kernels in ccl_kernels.cu run them with one CTA per tile and a
// __syncthreads() between phases.
//
// Method (PARemSP, arXiv 1606.05973):
//  * Section IV / Algorithm 7 split the image into chunks that are labelled
//    independently, each with its own label range, and then merge the chunk boundaries
//    with a concurrent Rem union (Algorithm 8).  Here the chunks are 2-D tiles of TH x TW
//    pixels, one per CTA, labelled in shared memory.
//  * Algorithm 6 (Scan_ARemSP) labels two rows at a time (e and g of Fig. 1b get one
//    label).  Here a tile is a stack of two-row strips; under 8-connectivity every
//    maximal run of columns that holds an object pixel in either row of a strip is
//    connected (vertical and diagonal neighbours inside the strip), so each such
//    "strip run" is one union-find node.
//  * Algorithm 2 (merge, Rem's union with splicing) joins nodes; the lock of Algorithm 8
//    becomes a compare-and-swap on the root, and every splice is also a compare-and-swap
//    of exactly the parent value the thread read (an unconditional splice, or an atomic
//    minimum, can overwrite a link another thread has just made and lose a union; see
//    rem_unite_g).  Links always go from the larger index to the smaller one, so the root
//    of every set is its smallest index (the invariant p[x] <= x of Algorithm 2).
//  * Runs are numbered per strip in column order, so the run covering a pixel is found
//    with one popcount.  Links go from the larger number to the smaller, so a local root
//    is the top-left run of its component; the component's raster-first pixel lies in
//    that run's strip and is found with an atomic minimum over the runs there.
//  * Local roots get global ids whose order is raster order ((row, tile column) segment,
//    then rank in the segment), so the global Rem union again makes every component's
//    root its raster-first pixel, which fixes the canonical numbering (background 0,
//    components 1..K in raster order of first pixels).
//  * Algorithm 3 (flatten) and the labelling pass become: count global roots per
//    (image row, tile column) segment, exclusive-scan the counts in raster order, give
//    each root its rank + 1, and write every pixel's label.  The first kernel stores one
//    16-bit root code per strip run, so the final kernel only maps runs to labels.
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define CCL_HD __host__ __device__ __forceinline__
#else
#define CCL_HD inline
#endif
#if defined(__CUDA_ARCH__)
#define CCL_UNROLL _Pragma("unroll")
#else
#define CCL_UNROLL
#endif

// Host builds of these functions exist only for the test emulator (tests/emu), which runs
// every CTA with one OS thread per CUDA thread; it provides the emu_* hooks below.
#if !defined(__CUDA_ARCH__)
void emu_cta_sync();
void emu_grid_sync();
void emu_yield();
uint32_t emu_ballot(bool p);
int emu_shfl(int v, int src, int width);
int emu_shfl_up(int v, int delta, int width);
int emu_lane();
#endif

#ifndef CCL_REFILL
#define CCL_REFILL 2
#endif
// L2 prefetch of the successor tile's inputs in the tile pass and in the final pass (1: its
// bit pack, 2: also its run codes), for launches that set Img::pf_dist
#ifndef CCL_PF_TILE
#define CCL_PF_TILE 1
#endif
#ifndef CCL_PF_FINAL
#define CCL_PF_FINAL 1
#endif

namespace ccl {

// ---- flags and sentinels ---------------------------------------------------------------
// device status word bits (ccl.h exposes them as CCL_STATUS_*)
constexpr int ST_LOOP_CAP = 1;   // a union-find loop exceeded its iteration cap
constexpr int ST_BOUNDS = 2;     // a checked index was out of range (debug builds)
constexpr int ST_BAD_VALUE = 4;  // a value that cannot occur was read (debug builds)
constexpr int ST_BARRIER = 8;    // a grid barrier gave up waiting (should never happen)

constexpr int SMEM_LOOP_CAP = 1 << 20;
constexpr int GLOBAL_LOOP_CAP = 1 << 24;

// ---- CTA / warp primitives ------------------------------------------------------------------
CCL_HD void cta_sync()
{
#if defined(__CUDA_ARCH__)
    __syncthreads();
#else
    emu_cta_sync();
#endif
}
CCL_HD int lane_id()
{
#if defined(__CUDA_ARCH__)
    return (int)(threadIdx.x & 31);
#else
    return emu_lane();
#endif
}
// number of threads of the CTA for which p holds; every thread of the CTA calls it (it is a
// barrier).  The emulator counts in *slot, a shared int no other thread uses meanwhile.
CCL_HD int cta_count(bool p, int *slot, int tid)
{
#if defined(__CUDA_ARCH__)
    (void)slot;
    (void)tid;
    return __syncthreads_count(p ? 1 : 0);
#else
    if (tid == 0)
        __atomic_store_n(slot, 0, __ATOMIC_SEQ_CST);
    emu_cta_sync();
    if (p)
        __atomic_fetch_add(slot, 1, __ATOMIC_SEQ_CST);
    emu_cta_sync();
    const int n = __atomic_load_n(slot, __ATOMIC_SEQ_CST);
    emu_cta_sync();
    return n;
#endif
}
// all 32 lanes of the warp must call these together
CCL_HD void warp_sync()
{
#if defined(__CUDA_ARCH__)
    __syncwarp();
#else
    (void)emu_ballot(true);
#endif
}
CCL_HD uint32_t warp_ballot(bool p)
{
#if defined(__CUDA_ARCH__)
    return __ballot_sync(0xFFFFFFFFu, p);
#else
    return emu_ballot(p);
#endif
}
CCL_HD int warp_shfl(int v, int src, int width = 32)
{
#if defined(__CUDA_ARCH__)
    return __shfl_sync(0xFFFFFFFFu, v, src, width);
#else
    return emu_shfl(v, src, width);
#endif
}
CCL_HD int warp_shfl_up(int v, int delta, int width = 32)
{
#if defined(__CUDA_ARCH__)
    return __shfl_up_sync(0xFFFFFFFFu, v, delta, width);
#else
    return emu_shfl_up(v, delta, width);
#endif
}
// inclusive sum over groups of `width` consecutive lanes (width a power of two <= 32)
CCL_HD int warp_incl_sum(int v, int width)
{
    const int lw = lane_id() & (width - 1);
    for (int d = 1; d < width; d <<= 1) {
        const int t = warp_shfl_up(v, d, width);
        if (lw >= d)
            v += t;
    }
    return v;
}

// ---- portable bit and atomic helpers ---------------------------------------------------
CCL_HD int popc32(uint32_t v)
{
#if defined(__CUDA_ARCH__)
    return __popc(v);
#else
    return __builtin_popcount(v);
#endif
}
CCL_HD int msb32(uint32_t v)  // v != 0
{
#if defined(__CUDA_ARCH__)
    return 31 - __clz(v);
#else
    return 31 - __builtin_clz(v);
#endif
}
CCL_HD int ctz32(uint32_t v)  // 32 for v == 0
{
#if defined(__CUDA_ARCH__)
    return v ? __ffs((int)v) - 1 : 32;
#else
    return v ? __builtin_ctz(v) : 32;
#endif
}
CCL_HD uint32_t mask_le(int b) { return b >= 31 ? 0xFFFFFFFFu : ((2u << b) - 1u); }
// bits 0..b set; b = -1 gives 0
CCL_HD uint32_t mask_upto(int b) { return b < 0 ? 0u : (b >= 31 ? 0xFFFFFFFFu : ((2u << b) - 1u)); }
CCL_HD uint32_t mask_lt(int b) { return b <= 0 ? 0u : (b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u)); }
CCL_HD int imin(int a, int b) { return a < b ? a : b; }

CCL_HD int at_cas(int *a, int cmp, int val)
{
#if defined(__CUDA_ARCH__)
    return atomicCAS(a, cmp, val);
#else
    emu_yield();
    __atomic_compare_exchange_n(a, &cmp, val, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST);
    return cmp;
#endif
}
CCL_HD int at_add(int *a, int v)
{
#if defined(__CUDA_ARCH__)
    return atomicAdd(a, v);
#else
    emu_yield();
    return __atomic_fetch_add(a, v, __ATOMIC_SEQ_CST);
#endif
}
CCL_HD void at_or(uint32_t *a, uint32_t v)
{
#if defined(__CUDA_ARCH__)
    atomicOr(a, v);
#else
    __atomic_fetch_or(a, v, __ATOMIC_SEQ_CST);
#endif
}
CCL_HD void flag_status(int *st, int f)
{
#if defined(__CUDA_ARCH__)
    atomicOr(st, f);
#else
    __atomic_fetch_or(st, f, __ATOMIC_SEQ_CST);
#endif
}
CCL_HD uint32_t at_cas_u(uint32_t *a, uint32_t cmp, uint32_t val)
{
#if defined(__CUDA_ARCH__)
    return atomicCAS(a, cmp, val);
#else
    emu_yield();
    __atomic_compare_exchange_n(a, &cmp, val, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST);
    return cmp;
#endif
}
CCL_HD void at_min_u(uint32_t *a, uint32_t v)
{
#if defined(__CUDA_ARCH__)
    atomicMin(a, v);
#else
    emu_yield();
    uint32_t cur = __atomic_load_n(a, __ATOMIC_SEQ_CST);
    while (v < cur && !__atomic_compare_exchange_n(a, &cur, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {
    }
#endif
}
// shared memory written by other threads of the CTA in the same phase: a fresh read every
// time (no register caching across loop iterations)
CCL_HD uint32_t ld_su(const uint32_t *a)
{
#if defined(__CUDA_ARCH__)
    return *(const volatile uint32_t *)a;
#else
    return __atomic_load_n(a, __ATOMIC_RELAXED);
#endif
}
CCL_HD void st_su(uint32_t *a, uint32_t v)
{
#if defined(__CUDA_ARCH__)
    *a = v;
#else
    __atomic_store_n(a, v, __ATOMIC_RELAXED);
#endif
}
CCL_HD int ld_s(const int *a)
{
#if defined(__CUDA_ARCH__)
    return *(const volatile int *)a;
#else
    return __atomic_load_n(a, __ATOMIC_RELAXED);
#endif
}
// Global memory that other CTAs of the same launch write (union-find parents, CTA sums,
// round flags).  These are strong relaxed accesses at GPU scope, not weak ones: a weak
// load of a parent word may return a value older than a link another CTA made before the
// last grid barrier (observed on GB300 for about 2% of labellings of large near-critical
// images as a root whose link was then overwritten by its label), whereas a strong load
// returns the coherent value, and the grid barrier's fences order them.
CCL_HD int ld_g(const int *a)
{
#if defined(__CUDA_ARCH__)
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
#else
    return __atomic_load_n(a, __ATOMIC_RELAXED);
#endif
}
// A hint to bring the 128-byte line holding p into L2 ahead of its use; callers pass only
// addresses inside their buffers.  No effect on results.  The host emulation reads the
// byte instead, so that an address sanitizer checks the address.
CCL_HD void prefetch_l2(const void *p)
{
#if defined(__CUDA_ARCH__)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
#else
    const volatile char c = *static_cast<const volatile char *>(p);
    (void)c;
#endif
}
// four consecutive ints from a 16-byte aligned address (one strong vector load; each
// element is read atomically, the four together are not)
CCL_HD void ld_g4(const int *a, int v[4])
{
#if defined(__CUDA_ARCH__)
    asm volatile("ld.relaxed.gpu.global.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "l"(a)
                 : "memory");
#else
    for (int k = 0; k < 4; k++)
        v[k] = __atomic_load_n(a + k, __ATOMIC_RELAXED);
#endif
}
CCL_HD void st_g(int *a, int v)
{
#if defined(__CUDA_ARCH__)
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
#else
    __atomic_store_n(a, v, __ATOMIC_RELAXED);
#endif
}

#if defined(CCL_DEBUG)
template <class I> CCL_HD I chk(I i, I n, int *st)
{
    if (i < 0 || i >= n) {
        flag_status(st, ST_BOUNDS);
        return 0;
    }
    return i;
}
#define CCL_CHK(i, n, st) ::ccl::chk((i), (n), (st))
#else
#define CCL_CHK(i, n, st) (i)
#endif

// 4 bytes -> 4 object bits, bit i = (byte i > T), with c = (255 - T) in every byte.
// x > T exactly when x + (255 - T) carries out of the byte; that carry is the majority of
// bit 7 of x, bit 7 of c and the carry into bit 7, computed without crossing bytes.  With
// T = 0 (c = 0xFF) this is the non-zero test.
CCL_HD uint32_t gt_nibble(uint32_t v, uint32_t c)
{
    const uint32_t t = (v & 0x7F7F7F7Fu) + (c & 0x7F7F7F7Fu);  // bit 7: carry into bit 7
    const uint32_t m = ((v & c) | ((v | c) & t)) & 0x80808080u;
    // gather bits 0, 8, 16, 24 of (m >> 7) into bits 28..31 (cross terms land elsewhere)
    return ((m >> 7) * 0x10204080u) >> 28;
}
// 4 bytes -> 4 bits, bit i = (byte i of a == byte i of b): a zero-byte test of a ^ b
// (bit 7 of a byte of ~((t & 0x7F..) + 0x7F..) | t) is clear exactly when the byte of t is 0)
CCL_HD uint32_t eq_nibble(uint32_t a, uint32_t b)
{
    const uint32_t t = a ^ b;
    const uint32_t m = ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
    return ((m >> 7) * 0x10204080u) >> 28;
}
// 16 bytes -> 16 object bits (bit i = byte i > T), c as in gt_nibble.  NZ: T = 0 (c is all
// ones), which the compiler then folds to the plain non-zero test.
template <bool NZ = false> CCL_HD uint32_t gt_mask16(const uint8_t *src, uint32_t c)
{
    if (NZ)
        c = 0xFFFFFFFFu;
    uint32_t v[4];
#if defined(__CUDA_ARCH__)
    const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(src));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
#else
    memcpy(v, src, 16);
#endif
    return gt_nibble(v[0], c) | (gt_nibble(v[1], c) << 4) | (gt_nibble(v[2], c) << 8) | (gt_nibble(v[3], c) << 12);
}
CCL_HD void store4(int *dst, const int v[4])
{
#if defined(__CUDA_ARCH__)
    __stcs(reinterpret_cast<int4 *>(dst), make_int4(v[0], v[1], v[2], v[3]));
#else
    memcpy(dst, v, 16);
#endif
}

// ---- tile configuration ----------------------------------------------------------------
// CONN = 8: a strip is two rows (under 8-connectivity every run of row 2s | row 2s+1 is
// connected).  CONN = 4: a strip is one row (diagonal contacts do not connect).
// CLS: multi-class labelling (neighbours connect when their bytes are equal and non-zero);
// a strip is one row and a run also ends where the value changes.
template <int TH_, int TW_, int NT_, int CONN_ = 8, bool CLS_ = false> struct Cfg {
    static constexpr int TH = TH_;        // tile rows (even: whole strips)
    static constexpr int TW = TW_;        // tile columns (multiple of 32)
    static constexpr int NT = NT_;        // threads per CTA
    static constexpr int CONN = CONN_;    // 8 or 4
    static constexpr bool CLS = CLS_;     // multi-class
    static constexpr int RPS = (CONN == 8 && !CLS) ? 2 : 1;  // rows per strip
    static constexpr int NW = TW / 32;    // 32-bit words per tile row
    static constexpr int NS = TH / RPS;   // strips per tile
    static constexpr int CH = TW / 16;    // 16-byte chunks per tile row
    // max components whose first pixel is in one tile row, and max runs in one strip: runs
    // of one value are separated by background (TW/2); runs of different classes may touch
    static constexpr int ROWCAP = CLS ? TW : TW / 2;
    static constexpr int RC = CLS ? TW : TW / 2;
    static constexpr int RMAX = NS * RC;  // max strip runs in one tile
    static_assert(TW % 32 == 0 && TH % 2 == 0, "tile shape");
    static_assert(CONN == 8 || CONN == 4, "connectivity");
    static_assert(TH * ROWCAP <= 65536, "root codes must fit 16 bits");
    static_assert(TH * TW < 65535 && RMAX <= 65536, "positions and run numbers must fit 16 bits");
    static_assert(ROWCAP % 4 == 0, "segments are read four parents at a time");
};

// Per-image device arguments.  All workspace arrays are owned by the caller of the kernels.
struct Img {
    const uint8_t *img;  // H rows of `pitch` bytes; object = byte > thr
    int64_t pitch;
    int H, W;
    int thr;             // 0..255; 0 makes every non-zero byte an object pixel
    int vec_in;          // img 16-byte aligned and pitch % 16 == 0
    int nTX, nTY;        // tiles across / down
    uint32_t *bitpack;   // [H][nTX*NW] object bits, bit b of word w = column 32w+b
    uint32_t *cstart;    // multi-class only: [H][nTX*NW] run starts (a run ends where the value changes)
    uint16_t *runinfo;   // [tile][strip][RC] root code of each strip run (row*ROWCAP + j)
    int *P;              // global parents, index ((y*nTX + tx)*ROWCAP + j)
    int *nseg;           // [H*nTX] local components whose first pixel lies in (y, tx)
    int *cnt;            // [H*nTX] global roots per segment, then exclusive offsets
    int *edgeRow;        // [nTY][2][nTX*TW] node id of top (0) / bottom (1) tile rows, -1 = bg
    int *edgeCol;        // [nTX][2][nTY*TH] node id of left (0) / right (1) tile columns
    int *bsum;           // per-CTA root counts of the global kernel, then their offsets
    int *K;              // number of components (device)
    struct GridSync *gsync;  // grid barrier state of the global kernel (workspace header)
    int *labels;         // [H][W] int32 output
    int vec_out;         // labels 16-byte aligned and W % 4 == 0
    int label_base;      // subtracted from the global rank labels (batch: ranks before this image)
    int *status;         // device status word (ST_* bits)
    int64_t nP, nSeg, nRunInfo;  // array sizes (for checked builds)
    int pf_dist;         // > 0: a tile-pass or final-pass CTA prefetches into L2 the inputs of
                         // tile (its tile + pf_dist), the tile the CTA replacing it will take
};

// Workspace layout for one image (byte offsets, each 256-byte aligned).
struct Layout {
    int nTX, nTY;
    int64_t nSeg, nP, nBitWords, nEdgeRow, nEdgeCol, nBsum, nRunInfo;
    int64_t off_bitpack, off_runinfo, off_P, off_nseg, off_cnt, off_edgeRow, off_edgeCol, off_bsum, off_cstart, bytes;
};
constexpr int MAX_GLOBAL_CTAS = 4096;  // upper bound on the global kernel's grid

CCL_HD int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

template <class C> CCL_HD Layout plan_layout(int H, int W)
{
    Layout L;
    L.nTX = (W + C::TW - 1) / C::TW;
    L.nTY = (H + C::TH - 1) / C::TH;
    L.nSeg = (int64_t)H * L.nTX;
    L.nP = L.nSeg * C::ROWCAP;
    L.nBitWords = (int64_t)H * L.nTX * C::NW;
    L.nRunInfo = (int64_t)L.nTX * L.nTY * C::RMAX;
    L.nEdgeRow = (int64_t)L.nTY * 2 * L.nTX * C::TW;
    L.nEdgeCol = (int64_t)L.nTX * 2 * L.nTY * C::TH;
    L.nBsum = MAX_GLOBAL_CTAS;
    int64_t o = 0;
    L.off_bitpack = o; o = align256(o + L.nBitWords * 4);
    L.off_runinfo = o; o = align256(o + L.nRunInfo * 2);
    L.off_P = o; o = align256(o + L.nP * 4);
    L.off_nseg = o; o = align256(o + L.nSeg * 4);
    L.off_cnt = o; o = align256(o + L.nSeg * 4);
    L.off_edgeRow = o; o = align256(o + L.nEdgeRow * 4);
    L.off_edgeCol = o; o = align256(o + L.nEdgeCol * 4);
    L.off_bsum = o; o = align256(o + L.nBsum * 4);
    L.off_cstart = o; o = align256(o + (C::CLS ? L.nBitWords * 4 : 0));
    L.bytes = o;
    return L;
}

// ---- shared-memory tile state ------------------------------------------------------------
// Strip runs are numbered per strip in column order: run k of strip s is union-find node
// u = s*RC + k.  The run covering object column x of strip s is therefore
//   u = s*RC + (number of run starts of strip s at columns <= x) - 1,
// which needs only a popcount and a per-word prefix of start counts.
template <class C> struct SmemRuns {
    uint32_t bits[C::TH][C::NW];     // object bits of the tile (rows beyond H are 0)
    uint32_t starts[C::NS][C::NW];   // run starts of strip s (row 2s | row 2s+1, or row s)
    int rpre[C::NS][C::NW];          // run starts of strip s before word w
};
// A parent word holds the parent's run number in its low 16 bits.  The high 16 bits are
// all ones while runs are joined (so every comparison of two words compares parents), and
// a root's high half later receives its component's first pixel (tile raster position).
// multi-class tiles also keep the tile's bytes (load phase only) and, per row, which
// pixels have the same class as their up-left, up and up-right neighbours
template <class C, bool = C::CLS> struct SmemCls {};
template <class C> struct SmemCls<C, true> {
    uint32_t eq[3][C::TH][C::NW];    // bit x of eq[d+1][r]: byte(r, x) == byte(r-1, x+d) != 0
    uint8_t raw[C::TH][C::TW];       // the tile's bytes (0 outside the image)
};
template <class C> struct SmemL : SmemRuns<C>, SmemCls<C> {
    uint32_t par[C::RMAX];           // union-find parents (see above)
    int red;                         // cta_count's slot (host emulation only)
    uint32_t rootbits[C::TH][C::NW]; // first pixels of the local components (union phase: join lists)
    int rootpre[C::TH][C::NW];       // exclusive popcount prefix of rootbits along a row (idem)
    // more room for the join lists on tiles too small to hold 32 entries per warp there
    static constexpr int JSPARE = (32 * (C::NT / 32) > 2 * C::TH * C::NW) ? 32 * (C::NT / 32) - 2 * C::TH * C::NW : 1;
    uint32_t jspare[JSPARE];
};
template <class C> struct SmemF : SmemRuns<C> {
    // final label of strip run v at lab[v + 1]; the entry below run 0 and the three above
    // the last run pad the reads of write_labels (read, never used)
    int lab[C::RMAX + 4];
};

constexpr uint32_t PAR_HI = 0xFFFF0000u;
constexpr uint32_t PAR_LO = 0x0000FFFFu;

// Rem's union with splicing (Algorithm 2) made safe for concurrent threads (Algorithm 8).
// Both writes are compare-and-swaps of exactly the parent value this thread read: the
// locked "still a root? then link" step of Algorithm 8, and also its unlocked splice
// p[r] <- p[other].  A splice that overwrote a parent it had not read would detach r from
// a tree that another thread had just attached it to, and no thread would reconnect that
// tree (a lost union; seen on GB300 and reproduced by an interleaving search).  A failed
// compare-and-swap re-reads and retries from the same node.  The tile pass runs the same
// steps on packed shared-memory words (Tile::unions); this is the global parent table
// (ids are raster-ordered node ids).
CCL_HD void rem_unite_g(int *P, int64_t n, int x, int y, int *st)
{
    int rx = (int)CCL_CHK((int64_t)x, n, st), ry = (int)CCL_CHK((int64_t)y, n, st);
    (void)n;
    for (int it = 0; it < GLOBAL_LOOP_CAP; it++) {
        const int px = (int)CCL_CHK((int64_t)ld_g(&P[rx]), n, st);
        const int py = (int)CCL_CHK((int64_t)ld_g(&P[ry]), n, st);
        if (px == py)
            return;
        if (px > py) {
            if (at_cas(&P[rx], px, py) != px)
                continue;
            if (px == rx)
                return;
            rx = px;
        } else {
            if (at_cas(&P[ry], py, px) != py)
                continue;
            if (py == ry)
                return;
            ry = py;
        }
    }
    flag_status(st, ST_LOOP_CAP);
}

// root of run x (a run whose parent is itself)
CCL_HD int find_s(const uint32_t *par, int n, int x, int *st)
{
    (void)n;
    x = CCL_CHK(x, n, st);
    for (int it = 0; it < SMEM_LOOP_CAP; it++) {
        const int p = (int)(ld_su(&par[x]) & PAR_LO);
        if (p == x)
            return x;
        x = CCL_CHK(p, n, st);
    }
    flag_status(st, ST_LOOP_CAP);
    return x;
}

// read-only global load (P after flatten, run codes): may use the non-coherent cache
template <class T> CCL_HD T ld_ro(const T *a)
{
#if defined(__CUDA_ARCH__)
    return __ldg(a);
#else
    return *a;
#endif
}

template <class C> struct Tile {
    using SR = SmemRuns<C>;
    using SL = SmemL<C>;
    using SF = SmemF<C>;

    // -- phase: image bytes -> object bits; clear root bits; every parent starts as a root --
    CCL_HD static void load_image(const Img &a, SL &s, int ty, int tx, int tid)
    {
        if constexpr (C::CLS) {
            load_classes(a, s, ty, tx, tid);
            return;
        }
        const int y0 = ty * C::TH, x0 = tx * C::TW;
        uint16_t *half = reinterpret_cast<uint16_t *>(&s.bits[0][0]);
        constexpr int PER = (C::TH * C::CH + C::NT - 1) / C::NT;
        const bool full = a.vec_in && (y0 + C::TH <= a.H) && (x0 + C::TW <= a.W);
        const uint32_t c = (uint32_t)(255 - a.thr) * 0x01010101u;  // object = byte > thr
        if (full) {
            // interior tile: issue every 16-byte load before using any of them
            if (a.thr == 0)
                load_full<true, PER>(a, half, y0, x0, c, tid);
            else
                load_full<false, PER>(a, half, y0, x0, c, tid);
        } else {
            for (int q = tid; q < C::TH * C::CH; q += C::NT) {
                const int r = q / C::CH, cc = q % C::CH;
                const int y = y0 + r, x = x0 + 16 * cc;
                uint32_t m = 0;
                if (y < a.H && x < a.W) {
                    const uint8_t *src = a.img + (int64_t)y * a.pitch + x;
                    if (a.vec_in && x + 16 <= a.W) {
                        m = gt_mask16(src, c);
                    } else {
                        const int n = imin(16, a.W - x);
                        for (int i = 0; i < n; i++)
                            m |= ((int)src[i] > a.thr ? 1u : 0u) << i;
                    }
                }
                half[q] = (uint16_t)m;  // little-endian: half 2w is the low half of word w
            }
        }
    }

    // L2 prefetch of the image rows of tile t (nothing when pf_dist is 0 or t is past the
    // last tile)
    CCL_HD static void prefetch_image(const Img &a, int t, int tid)
    {
        if (a.pf_dist <= 0 || t >= a.nTX * a.nTY)
            return;
        const int y0 = (t / a.nTX) * C::TH, x0 = (t % a.nTX) * C::TW;
        constexpr int LPR = (C::TW + 127) / 128;  // 128-byte lines per tile row
        for (int q = tid; q < C::TH * LPR; q += C::NT) {
            const int y = y0 + q / LPR, x = x0 + 128 * (q % LPR);
            if (y < a.H && x < a.W)
                prefetch_l2(a.img + (int64_t)y * a.pitch + x);
        }
    }

    // L2 prefetch of the bit-pack rows of tile t (and, CCL_PF_FINAL 2, its run codes)
    CCL_HD static void prefetch_final(const Img &a, int t, int tid)
    {
        if (a.pf_dist <= 0 || t >= a.nTX * a.nTY)
            return;
        const int y0 = (t / a.nTX) * C::TH, tx = t % a.nTX;
        const int64_t WW = (int64_t)a.nTX * C::NW;
        constexpr int LPR = (C::NW * 4 + 127) / 128;
        for (int q = tid; q < C::TH * LPR; q += C::NT) {
            const int y = y0 + q / LPR;
            if (y < a.H)
                prefetch_l2(a.bitpack + (int64_t)y * WW + tx * C::NW + 32 * (q % LPR));
        }
#if CCL_PF_FINAL >= 2
        const uint16_t *ri = a.runinfo + (int64_t)t * C::RMAX;
        for (int q = tid; q < C::RMAX / 64; q += C::NT)
            prefetch_l2(ri + 64 * q);
#endif
    }

    template <bool NZ, int PER>
    CCL_HD static void load_full(const Img &a, uint16_t *half, int y0, int x0, uint32_t c, int tid)
    {
        uint32_t m[PER];
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const int q = tid + i * C::NT;
            m[i] = 0;
            if (q < C::TH * C::CH) {
                const int r = q / C::CH, cc = q % C::CH;
                m[i] = gt_mask16<NZ>(a.img + (int64_t)(y0 + r) * a.pitch + x0 + 16 * cc, c);
            }
        }
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const int q = tid + i * C::NT;
            if (q < C::TH * C::CH)
                half[q] = (uint16_t)m[i];
        }
    }

    // Multi-class load: the tile's bytes into shared memory, then per (row, word) the object
    // bits (non-zero bytes), the run starts (object, and not the same value as the pixel to
    // the left) and the same-class masks toward the row above.  Pixels outside the tile
    // count as different (the boundary merge joins across tiles).
    CCL_HD static void load_classes(const Img &a, SL &s, int ty, int tx, int tid)
    {
        if constexpr (C::CLS) {
            const int y0 = ty * C::TH, x0 = tx * C::TW;
            const bool full = a.vec_in && (y0 + C::TH <= a.H) && (x0 + C::TW <= a.W);
            for (int q = tid; q < C::TH * C::CH; q += C::NT) {
                const int r = q / C::CH, cc = q % C::CH;
                const int y = y0 + r, x = x0 + 16 * cc;
                uint8_t *dst = &s.raw[r][16 * cc];
                if (full) {
                    const uint8_t *src = a.img + (int64_t)y * a.pitch + x;
                    uint32_t v[4];
#if defined(__CUDA_ARCH__)
                    const uint4 qv = __ldcs(reinterpret_cast<const uint4 *>(src));
                    v[0] = qv.x;
                    v[1] = qv.y;
                    v[2] = qv.z;
                    v[3] = qv.w;
#else
                    memcpy(v, src, 16);
#endif
                    for (int k = 0; k < 4; k++)
                        reinterpret_cast<uint32_t *>(dst)[k] = v[k];
                } else {
                    for (int i = 0; i < 16; i++)
                        dst[i] = (y < a.H && x + i < a.W) ? a.img[(int64_t)y * a.pitch + x + i] : (uint8_t)0;
                }
            }
            cta_sync();
            for (int q = tid; q < C::TH * C::NW; q += C::NT) {
                const int r = q / C::NW, w = q % C::NW;
                // 32 bytes of row r and of row r-1 as words (byte i of word k = column 32w+4k+i),
                // and the bytes just outside them; a byte outside the tile reads as 0, which
                // equals no object byte
                const uint32_t *cur = reinterpret_cast<const uint32_t *>(&s.raw[r][32 * w]);
                const uint32_t *up = reinterpret_cast<const uint32_t *>(&s.raw[r > 0 ? r - 1 : 0][32 * w]);
                const uint32_t upm = r > 0 ? 0xFFFFFFFFu : 0u;
                const uint32_t lb = (w > 0) ? s.raw[r][32 * w - 1] : 0u;
                const uint32_t ulb = (w > 0 && r > 0) ? s.raw[r - 1][32 * w - 1] : 0u;
                const uint32_t urb = (w + 1 < C::NW && r > 0) ? s.raw[r - 1][32 * w + 32] : 0u;
                uint32_t obj = 0, eqL = 0, eqUL = 0, eqU = 0, eqUR = 0;
                uint32_t cprev = lb << 24, uprev = ulb << 24;  // the byte before word k, in byte 3
                CCL_UNROLL
                for (int k = 0; k < 8; k++) {
                    const uint32_t v = cur[k], u = up[k] & upm;
                    const uint32_t un = (k < 7) ? (up[k + 1] & upm) : urb;
                    const uint32_t nz = gt_nibble(v, 0xFFFFFFFFu);
                    obj |= nz << (4 * k);
                    eqL |= (eq_nibble(v, (v << 8) | (cprev >> 24)) & nz) << (4 * k);
                    eqUL |= (eq_nibble(v, (u << 8) | (uprev >> 24)) & nz) << (4 * k);
                    eqU |= (eq_nibble(v, u) & nz) << (4 * k);
                    eqUR |= (eq_nibble(v, (u >> 8) | (un << 24)) & nz) << (4 * k);
                    cprev = v;
                    uprev = u;
                }
                s.bits[r][w] = obj;
                s.starts[r][w] = obj & ~eqL;
                s.eq[0][r][w] = eqUL;
                s.eq[1][r][w] = eqU;
                s.eq[2][r][w] = eqUR;
            }
        } else {
            (void)a;
            (void)s;
            (void)ty;
            (void)tx;
            (void)tid;
        }
    }

    CCL_HD static void store_bitpack(const Img &a, const SR &s, int ty, int tx, int tid)
    {
        const int y0 = ty * C::TH;
        const int64_t WW = (int64_t)a.nTX * C::NW;
        for (int q = tid; q < C::TH * C::NW; q += C::NT) {
            const int r = q / C::NW, w = q % C::NW;
            if (y0 + r < a.H) {
                const int64_t i = CCL_CHK((int64_t)(y0 + r) * WW + tx * C::NW + w, (int64_t)a.H * WW, a.status);
                a.bitpack[i] = s.bits[r][w];
                if constexpr (C::CLS)
                    a.cstart[i] = s.starts[r][w];
            }
        }
    }

    CCL_HD static void load_bitpack(const Img &a, SR &s, int ty, int tx, int tid)
    {
        const int y0 = ty * C::TH;
        const int64_t WW = (int64_t)a.nTX * C::NW;
        for (int q = tid; q < C::TH * C::NW; q += C::NT) {
            const int r = q / C::NW, w = q % C::NW;
            const bool in = y0 + r < a.H;
            const int64_t i = in ? CCL_CHK((int64_t)(y0 + r) * WW + tx * C::NW + w, (int64_t)a.H * WW, a.status) : 0;
            s.bits[r][w] = in ? ld_ro(&a.bitpack[i]) : 0u;
            if constexpr (C::CLS)
                s.starts[r][w] = in ? ld_ro(&a.cstart[i]) : 0u;
        }
    }

    CCL_HD static uint32_t strip_word(const SR &s, int st, int w)
    {
        if constexpr (C::RPS == 1)
            return s.bits[st][w];
        else
            return s.bits[2 * st][w] | s.bits[2 * st + 1][w];
    }

    // Tile raster position of the first pixel (raster order) of the strip run that starts
    // at bit b of word w: the first object pixel of the upper row inside the run if any,
    // else the run's first column in the lower row.
    CCL_HD static int first_pixel(const SR &s, int st, int w, int b)
    {
        if constexpr (C::RPS == 1)
            return st * C::TW + w * 32 + b;  // a one-row run starts at its first pixel
        else
            return first_pixel2(s, st, w, b);
    }

    CCL_HD static int first_pixel2(const SR &s, int st, int w, int b)
    {
        const uint32_t R0 = s.bits[2 * st][w];
        const uint32_t M = R0 | s.bits[2 * st + 1][w];
        const int x0 = w * 32 + b;
        const int len = ctz32(~(M >> b));  // <= 32 - b
        const uint32_t rm = (len >= 32) ? 0xFFFFFFFFu : (((1u << len) - 1u) << b);
        const uint32_t hit = R0 & rm;
        if (hit)
            return 2 * st * C::TW + w * 32 + ctz32(hit);
        if (b + len < 32)
            return (2 * st + 1) * C::TW + x0;
        for (int w2 = w + 1; w2 < C::NW; w2++) {
            const uint32_t R0b = s.bits[2 * st][w2];
            const uint32_t Mb = R0b | s.bits[2 * st + 1][w2];
            const int l2 = ctz32(~Mb);
            const uint32_t rm2 = (l2 >= 32) ? 0xFFFFFFFFu : ((1u << l2) - 1u);
            const uint32_t h2 = R0b & rm2;
            if (h2)
                return 2 * st * C::TW + w2 * 32 + ctz32(h2);
            if (l2 < 32)
                break;
        }
        return (2 * st + 1) * C::TW + x0;
    }

    CCL_HD static uint32_t starts_of(const SR &s, int st, int w)
    {
        const uint32_t M = strip_word(s, st, w);
        const uint32_t prev = (w > 0) ? (strip_word(s, st, w - 1) >> 31) : 0u;
        return M & ~((M << 1) | prev);
    }

    // -- phase: strip run starts, and how many runs of the strip start before each word.
    // The NW words of a strip sit in NW consecutive lanes, so the prefix is a shuffle scan.
    // The tile pass also makes every run it numbers a union-find root here (par holds an
    // entry only for runs that exist; no phase reads the entry of a run that does not).
    CCL_HD static void strip_runs(SL &s, int tid) { strip_runs_t<true>(s, s.par, tid); }
    CCL_HD static void strip_runs(SF &s, int tid) { strip_runs_t<false>(s, nullptr, tid); }

    template <bool INIT> CCL_HD static void strip_runs_t(SR &s, uint32_t *par, int tid)
    {
        static_assert(32 % C::NW == 0 && C::NT % 32 == 0, "a strip's words must share a warp");
        for (int u0 = 0; u0 < C::NS * C::NW; u0 += C::NT) {
            const int u = u0 + tid;
            const bool ok = u < C::NS * C::NW;
            const int st = ok ? u / C::NW : 0, w = u % C::NW;
            // multi-class run starts come from the bytes (load phase, or the global copy)
            const uint32_t st_bits = ok ? (C::CLS ? s.starts[st][w] : starts_of(s, st, w)) : 0u;
            const int c = popc32(st_bits);
            const int incl = warp_incl_sum(c, C::NW);
            if (ok) {
                s.starts[st][w] = st_bits;
                s.rpre[st][w] = incl - c;
                if constexpr (INIT) {
                    const int v0 = st * C::RC + incl - c;
                    for (int k = 0; k < c; k++)
                        par[v0 + k] = PAR_HI | (uint32_t)(v0 + k);
                }
            }
        }
    }

    // union-find node of the strip run covering object column x of strip st
    CCL_HD static int node(const SR &s, int st, int x)
    {
        const int w = x >> 5, b = x & 31;
        return st * C::RC + s.rpre[st][w] + popc32(s.starts[st][w] & mask_le(b)) - 1;
    }

    // -- phase: join strip runs that touch across strip boundaries ------------------------
    // Rows A = 2s-1 (last row of strip s-1) and B = 2s (first row of strip s).  Every pair
    // of single-row runs (one in A, one in B) that are 8-adjacent is found exactly once:
    // either the B run starts where A has a pixel at that column or one to the left, or
    // the A run starts one column right of a B pixel.
    // Multi-class: rows A = st-1 and B = st, and for each direction d (up-left, up,
    // up-right) the columns x where byte(B, x) == byte(A, x+d) != 0.  Every such contact
    // joins the B run covering x with the A run covering x+d; a contact is an event unless
    // the contact one column to the left (same d) joins the same two runs.
    // The joins of unit u (strip boundary u / NW, word u % NW), as two event masks, with
    // what is needed to turn an event into the two runs it joins.
    // Rows A = last row of strip st-1 and B = first row of strip st.  Every pair of
    // single-row runs (one in A, one in B) that are adjacent is found exactly once:
    // 8: the B run starts where A has a pixel at that column or one to the left, or the A
    //    run starts one column right of a B pixel;
    // 4: the B run starts under an A pixel, or the A run starts over a B pixel that does
    //    not start a B run.
    // The run of strip s covering bit b of the word (b = -1: the last bit of the word to
    // the left) is base + popcount(starts & bits 0..b).
    struct UnitEvents {
        uint32_t ev1 = 0, ev2 = 0, A = 0, sA = 0, sB = 0;
        int baseA = 0, baseB = 0;
    };

    // Events of a word that can join a new pair of strip runs.  Both runs an event at
    // column x joins cover a column in x-1..x, so two consecutive events y < x join the
    // same two strip runs when neither strip has a run start in columns y..x; such an x
    // is dropped (the kept event before it joins that pair).  With S the run starts of
    // both strips, x is kept when flag(x) holds:
    //   flag(x) = S(x) | (S(x-1) & E(x-1)) | (flag(x-1) & !E(x-1)),  flag(-1) = 1,
    // a carry chain (generate G = S | (S & E) << 1, propagate = no event one column to
    // the left), so one 64-bit addition evaluates it for all 32 columns.  Bit j of the
    // 64-bit words stands for column j - 1.
    CCL_HD static uint32_t new_pair_events(uint32_t E, uint32_t S)
    {
        const uint64_t G = ((uint64_t)(S | ((S & E) << 1)) << 1) | 1u;
        const uint64_t P = ~((uint64_t)E << 2);
        const uint64_t A = G | P;
        const uint64_t carry = (A + G) ^ A ^ G;  // carry into bit j = flag(column j - 2)
        return E & (uint32_t)(carry >> 2);
    }
    CCL_HD static UnitEvents unit_events(const SL &s, int u)
    {
        UnitEvents e;
        const int st = u / C::NW, w = u % C::NW;
        if (u < C::NS * C::NW && st > 0) {
            const int ra = C::RPS * st - 1, rb = C::RPS * st;
            e.A = s.bits[ra][w];
            const uint32_t B = s.bits[rb][w];
            const uint32_t Ap = (w > 0) ? (s.bits[ra][w - 1] >> 31) : 0u;
            const uint32_t Bp = (w > 0) ? (s.bits[rb][w - 1] >> 31) : 0u;
            const uint32_t Ash = (e.A << 1) | Ap, Bsh = (B << 1) | Bp;
            const uint32_t sBr = B & ~Bsh, sAr = e.A & ~Ash;  // single-row run starts
            e.ev1 = (C::CONN == 8) ? (sBr & (e.A | Ash)) : (sBr & e.A);
            e.ev2 = (C::CONN == 8) ? (sAr & Bsh) : (sAr & B & ~sBr);
            e.sA = s.starts[st - 1][w];
            e.sB = s.starts[st][w];
            const uint32_t keep = new_pair_events(e.ev1 | e.ev2, e.sA | e.sB);
            e.ev1 &= keep;
            e.ev2 &= keep;
            e.baseA = (st - 1) * C::RC + s.rpre[st - 1][w] - 1;
            e.baseB = st * C::RC + s.rpre[st][w] - 1;
        }
        return e;
    }

    CCL_HD static void unions_cls(const Img &a, SL &s, int tid)
    {
        if constexpr (C::CLS) {
            for (int u0 = 0; u0 < C::NS * C::NW; u0 += C::NT) {
                const int u = u0 + tid, st = u / C::NW, w = u % C::NW;
                uint32_t ev[3] = {0u, 0u, 0u}, sA = 0, sB = 0, sAn = 0;
                int baseA = 0, baseB = 0, baseAn = 0;
                if (u < C::NS * C::NW && st > 0) {
                    sA = s.starts[st - 1][w];
                    sB = s.starts[st][w];
                    const uint32_t sAp = (w > 0) ? s.starts[st - 1][w - 1] : 0u;
                    sAn = (w + 1 < C::NW) ? s.starts[st - 1][w + 1] : 0u;
                    baseA = (st - 1) * C::RC + s.rpre[st - 1][w] - 1;
                    baseB = st * C::RC + s.rpre[st][w] - 1;
                    baseAn = (w + 1 < C::NW) ? (st - 1) * C::RC + s.rpre[st - 1][w + 1] - 1 : 0;
                    // A starts seen from column x: at x-1, x, x+1
                    const uint32_t SA[3] = {(sA << 1) | (sAp >> 31), sA, (sA >> 1) | (sAn << 31)};
                    for (int d = 0; d < 3; d++) {
                        if (C::CONN == 4 && d != 1)
                            continue;
                        const uint32_t M = s.eq[d][st][w];
                        ev[d] = M & ~((M << 1) & ~sB & ~SA[d]);
                    }
                }
                int rx = -1, ry = -1;
                for (int it = 0;; it++) {
                    if (rx < 0 && (ev[0] | ev[1] | ev[2])) {
                        const int d = ev[0] ? 0 : (ev[1] ? 1 : 2);
                        const int b = ctz32(ev[d]);
                        ev[d] &= ev[d] - 1u;
                        const int nb = baseB + popc32(sB & mask_upto(b));
                        const int xa = b + d - 1;  // column of the A pixel, -1..32
                        const int na = (xa < 32) ? baseA + popc32(sA & mask_upto(xa)) : baseAn + (int)(sAn & 1u);
                        rx = CCL_CHK(nb, C::RMAX, a.status);
                        ry = CCL_CHK(na, C::RMAX, a.status);
                    }
                    if (!warp_ballot(rx >= 0 || (ev[0] | ev[1] | ev[2]) != 0u))
                        break;
                    if (it == SMEM_LOOP_CAP) {
                        flag_status(a.status, ST_LOOP_CAP);
                        break;
                    }
                    if (rx >= 0) {
                        const uint32_t px = ld_su(&s.par[rx]);
                        const uint32_t py = ld_su(&s.par[ry]);
                        const bool xs = px > py;
                        const int r = xs ? rx : ry;
                        const uint32_t pr = xs ? px : py, po = xs ? py : px;
                        if (px == py) {
                            rx = -1;
                        } else if (at_cas_u(&s.par[r], pr, po) == pr) {
                            const int up = CCL_CHK((int)(pr & PAR_LO), C::RMAX, a.status);
                            if (up == r)
                                rx = -1;
                            else if (xs)
                                rx = up;
                            else
                                ry = up;
                        }
                    }
                }
            }
        } else {
            (void)a;
            (void)s;
            (void)tid;
        }
    }

    CCL_HD static void unions(const Img &a, SL &s, int tid)
    {
        if constexpr (C::CLS)
            unions_cls(a, s, tid);
        else
            unions_bin(a, s, tid);
    }

    // The joins of a warp's units go through a list in shared memory (the root arrays,
    // unused until the roots phase): rounds append every lane's next event (its r-th), so
    // neighbouring entries come from different units, and in every pass each lane without
    // a join in progress takes the next listed one.  Lanes stay busy until the warp's
    // joins run out, instead of idling once their own unit's events are done.
    static constexpr int JCAP = (2 * C::TH * C::NW + SL::JSPARE) / (C::NT / 32);
    // events a lane lists per refill round (fewer rounds, fewer votes)
    static constexpr int REFILL = (JCAP >= 64 * CCL_REFILL) ? CCL_REFILL : 1;
    static_assert(JCAP >= 32, "join list too short");

    CCL_HD static void unions_bin(const Img &a, SL &s, int tid)
    {
        // the lists span rootbits, rootpre and jspare: members of 4-byte elements declared
        // one after another, so they are contiguous
        uint32_t *jl = reinterpret_cast<uint32_t *>(&s.rootbits[0][0]) + (tid / 32) * JCAP;
        const uint32_t lt = mask_lt(lane_id());
        // every thread runs the same number of outer passes (NT is a multiple of 32), so
        // whole warps reach the votes below
        for (int u0 = 0; u0 < C::NS * C::NW; u0 += C::NT) {
            const UnitEvents e = unit_events(s, u0 + tid);
            uint32_t ev1 = e.ev1, ev2 = e.ev2;
            if (!warp_ballot((ev1 | ev2) != 0u))
                continue;  // no joins in this warp's units
            const uint32_t A = e.A, sA = e.sA, sB = e.sB;
            const int baseA = e.baseA, baseB = e.baseB;
            // An event at bit b joins the A run covering column b or b-1 with the B run
            // covering b or b-1; with m = 1 << b, the runs covering b and b-1 are counted
            // by the masks m | (m - 1) and m - 1 (b = 0: the word to the left).  An event
            // that joins the same two runs as the lane's previous one is not listed.
            uint32_t last = 0xFFFFFFFFu;
            int head = 0, tail = 0;  // the warp's list: entries [head, tail) not yet taken
            bool unlisted = true;    // some lane has events not yet listed (warp-uniform)
            int rx = -1, ry = -1;
            for (int it = 0;; it++) {
                if (head == tail && unlisted) {
                    // refill: every lane's next REFILL events per round, the round's first
                    // events of all lanes before its second ones
                    warp_sync();  // the old entries have all been read
                    head = tail = 0;
                    for (;;) {
                        uint32_t key[REFILL];
                        bool has[REFILL];
                        CCL_UNROLL
                        for (int q = 0; q < REFILL; q++) {
                            has[q] = (ev1 | ev2) != 0u;
                            key[q] = 0;
                            if (has[q]) {
                                const uint32_t E = ev1 | ev2;
                                const uint32_t m = E & (0u - E);
                                const uint32_t below = m - 1u, upto = below | m;
                                const bool first = (ev1 & m) != 0u;  // an event of the first kind
                                ev1 &= ~m;
                                ev2 &= ~m;
                                const uint32_t mA = (C::CONN == 8 && first && !(A & m)) ? below : upto;
                                const uint32_t mB = (C::CONN == 8 && !first) ? below : upto;
                                const int na = baseA + popc32(sA & mA), nb = baseB + popc32(sB & mB);
                                key[q] = ((uint32_t)na << 16) | (uint32_t)nb;
                                has[q] = key[q] != last;
                                last = key[q];
                            }
                        }
                        CCL_UNROLL
                        for (int q = 0; q < REFILL; q++) {
                            const uint32_t mk = warp_ballot(has[q]);
                            if (has[q])
                                jl[tail + popc32(mk & lt)] = key[q];
                            tail += popc32(mk);
                        }
                        unlisted = warp_ballot((ev1 | ev2) != 0u) != 0u;
                        if (tail > JCAP - 32 * REFILL || !unlisted)
                            break;
                    }
                    warp_sync();  // the new entries are visible to every lane
                }
                // lanes without a join in progress take the next listed joins, in order
                const uint32_t fr = warp_ballot(rx < 0);
                const int avail = tail - head;
                if (rx < 0) {
                    const int r = popc32(fr & lt);
                    if (r < avail) {
                        const uint32_t key = jl[head + r];
                        rx = CCL_CHK((int)(key & PAR_LO), C::RMAX, a.status);
                        ry = CCL_CHK((int)(key >> 16), C::RMAX, a.status);
                    }
                }
                head += imin(popc32(fr), avail);
                // a lane is busy if it was already or has just taken an entry: with no lane
                // busy, nothing listed and nothing left to list, the warp is done
                if (fr == 0xFFFFFFFFu && avail == 0 && !unlisted)
                    break;
                if (it == SMEM_LOOP_CAP) {
                    flag_status(a.status, ST_LOOP_CAP);
                    break;
                }
                // one step of Rem's union (Algorithm 2 with Algorithm 8's compare-and-swap
                // writes, as in rem_unite_g)
                if (rx >= 0) {
                    const uint32_t px = ld_su(&s.par[rx]);
                    const uint32_t py = ld_su(&s.par[ry]);
                    const bool xs = px > py;  // write the larger parent's entry
                    const int r = xs ? rx : ry;
                    const uint32_t pr = xs ? px : py, po = xs ? py : px;
                    if (px == py) {
                        rx = -1;  // same parent: already joined
                    } else if (at_cas_u(&s.par[r], pr, po) == pr) {
                        const int up = CCL_CHK((int)(pr & PAR_LO), C::RMAX, a.status);
                        if (up == r)
                            rx = -1;  // a root was linked: this join is done
                        else if (xs)
                            rx = up;
                        else
                            ry = up;
                    }  // else: changed since read, read again in the next pass
                }
            }
        }
        warp_sync();
    }

    // -- phase: every run points at its root.  A component's first pixel lies in its
    // root's strip (the root is its top-left run), so the runs of that strip lower the
    // root's key (high half of its word) to the smallest first pixel among them.
    CCL_HD static void roots(const Img &a, SL &s, int tid)
    {
        // the root bits held the union phase's join lists: clear them for mark_roots (a
        // barrier separates this phase from mark_roots)
        for (int q = tid; q < C::TH * C::NW; q += C::NT)
            (&s.rootbits[0][0])[q] = 0u;
        for (int u = tid; u < C::NS * C::NW; u += C::NT) {
            const int st = u / C::NW, w = u % C::NW;
            uint32_t todo = s.starts[st][w];
            int v = st * C::RC + s.rpre[st][w];
            while (todo) {
                const int b = ctz32(todo);
                todo &= todo - 1u;
                const int r = find_s(s.par, C::RMAX, v, a.status);
                if (r != v)
                    st_su(&s.par[v], PAR_HI | (uint32_t)r);
                if (r / C::RC == st)
                    at_min_u(&s.par[r], ((uint32_t)first_pixel(s, st, w, b) << 16) | (uint32_t)r);
                v++;
            }
        }
    }

    // -- phase: mark each local component's first pixel ---------------------------------
    CCL_HD static void mark_roots(const Img &a, SL &s, int tid)
    {
        for (int u = tid; u < C::NS * C::NW; u += C::NT) {
            const int st = u / C::NW, w = u % C::NW;
            const int n = popc32(s.starts[st][w]);
            const int v0 = st * C::RC + s.rpre[st][w];
            for (int k = 0; k < n; k++) {
                const uint32_t p = s.par[v0 + k];
                if ((int)(p & PAR_LO) == v0 + k) {
                    const int pos = CCL_CHK((int)(p >> 16), C::TH * C::TW, a.status);
                    at_or(&s.rootbits[pos / C::TW][(pos % C::TW) >> 5], 1u << (pos & 31));
                }
            }
        }
    }

    // -- phase: rank of roots along each tile row; segment sizes --------------------------
    CCL_HD static void root_prefix(const Img &a, SL &s, int ty, int tx, int tid)
    {
        const int y0 = ty * C::TH;
        for (int q0 = 0; q0 < C::TH * C::NW; q0 += C::NT) {
            const int q = q0 + tid;
            const bool ok = q < C::TH * C::NW;
            const int r = ok ? q / C::NW : 0, w = q % C::NW;
            const int c = ok ? popc32(s.rootbits[r][w]) : 0;
            const int incl = warp_incl_sum(c, C::NW);
            if (ok) {
                s.rootpre[r][w] = incl - c;
                if (w == C::NW - 1 && y0 + r < a.H)
                    a.nseg[CCL_CHK((int64_t)(y0 + r) * a.nTX + tx, a.nSeg, a.status)] = incl;
            }
        }
    }

    // tile-local code (row * ROWCAP + j) of the component whose first pixel is `pos`
    CCL_HD static int code_of(const SL &s, int pos)
    {
        const int rr = pos / C::TW, cc = pos % C::TW;
        const int j = s.rootpre[rr][cc >> 5] + popc32(s.rootbits[rr][cc >> 5] & mask_lt(cc & 31));
        return rr * C::ROWCAP + j;
    }

    CCL_HD static int64_t gid_of_code(const Img &a, int ty, int tx, int code)
    {
        const int rr = code / C::ROWCAP, j = code % C::ROWCAP;
        return ((int64_t)(ty * C::TH + rr) * a.nTX + tx) * C::ROWCAP + j;
    }

    // first pixel of the component of run v (after the roots phase a run's parent is
    // its root, and a root's key is its component's first pixel)
    CCL_HD static int comp_pos(const Img &a, const SL &s, int v)
    {
        const int r = CCL_CHK((int)(s.par[v] & PAR_LO), C::RMAX, a.status);
        return CCL_CHK((int)(s.par[r] >> 16), C::TH * C::TW, a.status);
    }

    // -- phase: run codes for the final pass, one global node per local root, edge ids ------
    CCL_HD static void outputs(const Img &a, const SL &s, int ty, int tx, int tid)
    {
        const int64_t tbase = ((int64_t)ty * a.nTX + tx) * C::RMAX;
        for (int u = tid; u < C::NS * C::NW; u += C::NT) {
            const int st = u / C::NW, w = u % C::NW;
            const int n = popc32(s.starts[st][w]);
            const int v0 = st * C::RC + s.rpre[st][w];
            for (int k = 0; k < n; k++)
                a.runinfo[CCL_CHK(tbase + v0 + k, a.nRunInfo, a.status)] = (uint16_t)code_of(s, comp_pos(a, s, v0 + k));
        }
        for (int q = tid; q < C::TH * C::NW; q += C::NT) {
            const int r = q / C::NW, w = q % C::NW;
            uint32_t rb = s.rootbits[r][w];
            int64_t gid = ((int64_t)(ty * C::TH + r) * a.nTX + tx) * C::ROWCAP + s.rootpre[r][w];
            while (rb) {
                rb &= rb - 1u;
                a.P[CCL_CHK(gid, a.nP, a.status)] = (int)gid;
                gid++;
            }
        }
        const int64_t WP = (int64_t)a.nTX * C::TW, HP = (int64_t)a.nTY * C::TH;
        for (int x = tid; x < C::TW; x += C::NT) {
            a.edgeRow[CCL_CHK((int64_t)(2 * ty) * WP + tx * C::TW + x, (int64_t)a.nTY * 2 * WP, a.status)] =
                pixel_gid(a, s, ty, tx, 0, x);
            a.edgeRow[CCL_CHK((int64_t)(2 * ty + 1) * WP + tx * C::TW + x, (int64_t)a.nTY * 2 * WP, a.status)] =
                pixel_gid(a, s, ty, tx, C::TH - 1, x);
        }
        for (int r = tid; r < C::TH; r += C::NT) {
            a.edgeCol[CCL_CHK((int64_t)(2 * tx) * HP + ty * C::TH + r, (int64_t)a.nTX * 2 * HP, a.status)] =
                pixel_gid(a, s, ty, tx, r, 0);
            a.edgeCol[CCL_CHK((int64_t)(2 * tx + 1) * HP + ty * C::TH + r, (int64_t)a.nTX * 2 * HP, a.status)] =
                pixel_gid(a, s, ty, tx, r, C::TW - 1);
        }
    }

    CCL_HD static int pixel_gid(const Img &a, const SL &s, int ty, int tx, int r, int x)
    {
        if (!((s.bits[r][x >> 5] >> (x & 31)) & 1u))
            return -1;
        return (int)gid_of_code(a, ty, tx, code_of(s, comp_pos(a, s, node(s, r / C::RPS, x))));
    }

    // -- final pass: the label of every strip run, from its code and the global table ------
    // After flatten P[id] is either -(final label) (a global root) or the id of its global
    // root, whose entry holds -(final label).
    CCL_HD static void run_labels(const Img &a, SF &s, int ty, int tx, int tid)
    {
        const int64_t tbase = ((int64_t)ty * a.nTX + tx) * C::RMAX;
        for (int u = tid; u < C::NS * C::NW; u += C::NT) {
            const int st = u / C::NW, w = u % C::NW;
            const int n = popc32(s.starts[st][w]);
            const int v0 = st * C::RC + s.rpre[st][w];
            int prev_code = -1, prev_lab = 0;
            // four runs at a time: their codes, then their parents, then the roots' entries,
            // so one batch waits for three loads instead of three per run
            for (int k0 = 0; k0 < n; k0 += 4) {
                int code[4], v[4];
                bool fresh[4];
                for (int k = 0; k < 4; k++)
                    code[k] = (k0 + k < n) ? ld_ro(&a.runinfo[CCL_CHK(tbase + v0 + k0 + k, a.nRunInfo, a.status)]) : -1;
                for (int k = 0; k < 4; k++) {
                    fresh[k] = code[k] >= 0 && code[k] != ((k == 0) ? prev_code : code[k - 1]);
                    v[k] = fresh[k] ? ld_ro(&a.P[CCL_CHK(gid_of_code(a, ty, tx, code[k]), a.nP, a.status)]) : -1;
                }
                for (int k = 0; k < 4; k++)
                    if (v[k] >= 0)  // not a global root: its entry names the root, which holds -label
                        v[k] = ld_ro(&a.P[CCL_CHK((int64_t)v[k], a.nP, a.status)]);
                for (int k = 0; k < 4 && k0 + k < n; k++) {
                    if (fresh[k]) {
                        prev_lab = -v[k] - a.label_base;
#if defined(CCL_DEBUG)
                        if (prev_lab <= 0) {
                            flag_status(a.status, ST_BAD_VALUE);
                            prev_lab = 0;
                        }
#endif
                    }
                    s.lab[v0 + k0 + k + 1] = prev_lab;
                }
                prev_code = code[3 < n - k0 - 1 ? 3 : n - k0 - 1];
            }
        }
    }

    // One item: four columns x..x+3 of one strip, i.e. 4 pixels of each of its RPS rows.
    // With S the strip's run starts in word w and o = x % 32, the run covering column x + k
    // (if any) is i0 + c_k, where i0 counts the runs starting at or before x (rpre and a
    // popcount) and c_k the starts in columns x+1..x+k.  Runs of one strip are separated by
    // background (binary images), so c_k <= 2 and three label reads serve the item's 4 or 8
    // pixels; multi-class runs may touch (c_k <= k, four reads).
    CCL_HD static void write_labels(const Img &a, const SF &s, int ty, int tx, int tid)
    {
        const int y0 = ty * C::TH, x0 = tx * C::TW;
        constexpr int G = C::TW / 4;
        const bool full = a.vec_out && y0 + C::TH <= a.H && x0 + C::TW <= a.W;
        for (int q = tid; q < C::NS * G; q += C::NT) {
            const int st = q / G, x = (q % G) * 4;
            const int w = x >> 5, o = x & 31;
            const uint32_t S = s.starts[st][w];
            const uint32_t Sx = S >> o;
            // lab index (labels are stored one entry up) of the run at or before column x
            const int i0 = CCL_CHK(st * C::RC + s.rpre[st][w] + popc32(S & mask_le(o)), C::RMAX + 1, a.status);
            const int c1 = (int)((Sx >> 1) & 1u);
            const int c2 = c1 + (int)((Sx >> 2) & 1u);
            const int c3 = c2 + (int)((Sx >> 3) & 1u);
            const int L0 = s.lab[i0], L1 = s.lab[i0 + 1], L2 = s.lab[i0 + 2];
            int cand[4];
            cand[0] = L0;
            cand[1] = c1 ? L1 : L0;
            if constexpr (C::CLS) {
                const int L3 = s.lab[i0 + 3];
                cand[2] = c2 == 0 ? L0 : (c2 == 1 ? L1 : L2);
                cand[3] = c3 == 0 ? L0 : (c3 == 1 ? L1 : (c3 == 2 ? L2 : L3));
            } else {
                cand[2] = c2 ? L1 : L0;
                cand[3] = c3 == 0 ? L0 : (c3 == 1 ? L1 : L2);
            }
            CCL_UNROLL
            for (int rr = 0; rr < C::RPS; rr++) {
                const int r = C::RPS * st + rr;
                const int y = y0 + r, gx = x0 + x;
                const uint32_t R = s.bits[r][w] >> o;
                int v[4];
                CCL_UNROLL
                for (int k = 0; k < 4; k++)
                    v[k] = ((R >> k) & 1u) ? cand[k] : 0;
                int *dst = a.labels + (int64_t)y * a.W + gx;
                if (full) {
                    store4(dst, v);
                } else if (y < a.H && gx < a.W) {
                    if (a.vec_out && gx + 4 <= a.W) {
                        store4(dst, v);
                    } else {
                        for (int k = 0; k < 4; k++)
                            if (gx + k < a.W)
                                dst[k] = v[k];
                    }
                }
            }
        }
    }
};

// ---- boundary merge (between tiles), Algorithm 7's boundary loop -------------------------
// For an object pixel e on one side of a tile edge, with b the pixel facing it and a, c
// the two diagonal ones: join e with b if b is an object pixel, else with a and c.  A pair
// already joined through the previous pixel along the edge (same node id) is skipped.
struct EdgeItem {
    int e, b, aa, c;
    bool same_prev;
    int ce, cb, ca, cc;  // multi-class: the bytes of the four pixels
    int pe, pm2;         // multi-class: the previous pixel's node on e's side, and the node
                         // facing two pixels back (the previous pixel's other diagonal)
};

// Horizontal tile boundaries of binary images are merged from the bit pack in units of
// HUNIT columns (multi-class images, whose contacts depend on the bytes, keep one item per
// column).  Vertical boundaries take one item per row.
constexpr int HUNIT = 8;
template <class C> CCL_HD int64_t horizontal_items(int nTY, int W)
{
    return C::CLS ? (int64_t)(nTY - 1) * W : (int64_t)(nTY - 1) * ((W + HUNIT - 1) / HUNIT);
}
template <class C> CCL_HD int64_t edge_items(int nTX, int nTY, int H, int W)
{
    return horizontal_items<C>(nTY, W) + (int64_t)(nTX - 1) * H;
}

// item i < nh: horizontal boundary above band 1 + i / W at column i % W; else vertical
// boundary left of tile column 1 + k / H at row k % H (k = i - nh)
template <class C> CCL_HD EdgeItem load_edge_item(const Img &a, int64_t i, int64_t nh)
{
    EdgeItem it;
    if (i < nh) {
        const int ty = 1 + (int)(i / a.W), x = (int)(i % a.W);
        const int64_t WP = (int64_t)a.nTX * C::TW;
        const int *top = a.edgeRow + (int64_t)(2 * ty) * WP;
        const int *above = a.edgeRow + (int64_t)(2 * ty - 1) * WP;
        it.e = top[x];
        it.b = above[x];
        it.aa = (x > 0) ? above[x - 1] : -1;
        it.c = (x + 1 < a.W) ? above[x + 1] : -1;
        it.same_prev = (x > 0) && top[x - 1] == it.e;
        if constexpr (C::CLS) {
            const uint8_t *r0 = a.img + (int64_t)(ty * C::TH) * a.pitch, *r1 = r0 - a.pitch;
            it.ce = r0[x];
            it.cb = r1[x];
            it.ca = (x > 0) ? r1[x - 1] : -1;
            it.cc = (x + 1 < a.W) ? r1[x + 1] : -1;
            it.pe = (x > 0) ? top[x - 1] : -1;
            it.pm2 = (x > 1) ? above[x - 2] : -1;
        }
    } else {
        const int64_t k = i - nh;
        const int tx = 1 + (int)(k / a.H), y = (int)(k % a.H);
        const int64_t HP = (int64_t)a.nTY * C::TH;
        const int *left = a.edgeCol + (int64_t)(2 * tx - 1) * HP;
        const int *me = a.edgeCol + (int64_t)(2 * tx) * HP;
        const int yb0 = (y / C::TH) * C::TH;
        const int yb1 = imin(yb0 + C::TH, a.H);
        it.e = me[y];
        it.b = left[y];
        it.aa = (y - 1 >= yb0) ? left[y - 1] : -1;
        it.c = (y + 1 < yb1) ? left[y + 1] : -1;
        it.same_prev = (y - 1 >= yb0) && me[y - 1] == it.e;
        if constexpr (C::CLS) {
            const uint8_t *col = a.img + tx * C::TW;  // column tx*TW of row 0
            it.ce = col[(int64_t)y * a.pitch];
            it.cb = col[(int64_t)y * a.pitch - 1];
            it.ca = (y - 1 >= yb0) ? col[(int64_t)(y - 1) * a.pitch - 1] : -1;
            it.cc = (y + 1 < yb1) ? col[(int64_t)(y + 1) * a.pitch - 1] : -1;
            it.pe = (y - 1 >= yb0) ? me[y - 1] : -1;
            it.pm2 = (y - 2 >= yb0) ? left[y - 2] : -1;
        }
    }
    return it;
}

// the union of two global node ids in the global parent table
struct UniteGlobal {
    const Img &a;
    CCL_HD void operator()(int x, int y) const { rem_unite_g(a.P, a.nP, x, y, a.status); }
};

template <class C, class U> CCL_HD void apply_edge_item(const Img &a, const EdgeItem &it, const U &unite)
{
    if (it.e < 0)
        return;
    if constexpr (C::CLS) {
        // multi-class: join each facing pixel (and, under 8-connectivity, each diagonal one)
        // of the same value.  A node has one value, so a pair is the same pair as one the
        // previous pixel along the edge formed when that pixel has the same node e and n is
        // one of its facing nodes (two back, one back, this one); that pair was joined there
        // (or skipped the same way, back to where it was joined).
        const bool prev = it.pe == it.e;
        auto fresh = [&](int n) {
            return !(prev && (n == it.b || n == it.aa || (C::CONN == 8 && n == it.pm2)));
        };
        const bool jb = it.b >= 0 && it.cb == it.ce;
        if (jb && (C::CONN == 8 ? fresh(it.b) : !(prev && it.b == it.aa)))
            unite(it.e, it.b);
        if (C::CONN == 8) {
            const bool ja = it.aa >= 0 && it.ca == it.ce && !(jb && it.aa == it.b);
            if (ja && fresh(it.aa))
                unite(it.e, it.aa);
            const bool jc = it.c >= 0 && it.cc == it.ce && !(jb && it.c == it.b) &&
                            !(it.aa >= 0 && it.ca == it.ce && it.c == it.aa);
            if (jc && fresh(it.c))
                unite(it.e, it.c);
        }
        return;
    }
    if constexpr (C::CONN == 4) {
        // 4-connectivity: only the facing pixel; the previous edge pixel (same node) has
        // already joined through its own facing pixel if that one is an object pixel
        if (it.b >= 0 && !(it.same_prev && it.aa >= 0))
            unite(it.e, it.b);
        return;
    }
    if (it.b >= 0) {
        if (!it.same_prev)
            unite(it.e, it.b);
    } else {
        if (it.aa >= 0 && !it.same_prev)
            unite(it.e, it.aa);
        if (it.c >= 0)
            unite(it.e, it.c);
    }
}

// Unit u of the horizontal boundaries (binary images): the boundary above tile row
// 1 + u / per, columns x0 .. x0 + HUNIT - 1.  Rows A (the last row of the tile row above) and
// B (the first row of the tile row below) come from the bit pack as windows of 32 columns
// starting at x0 - 1 (bit j = column x0 - 1 + j).  Every pair of single-row runs, one in A
// and one in B, that touch is found once, at the column where the later of the two starts,
// as the tile pass finds them between strips (8: the B run starts where A has a pixel at
// that column or one to the left, or the A run starts one column right of a B pixel;
// 4: the B run starts under an A pixel, or the A run starts over a B pixel that does not
// start a B run).  Each pair is joined through the node ids of its two touching pixels
// (the tile-edge ids); a pair with the same two ids as the unit's previous one is skipped.
template <class C, class U> CCL_HD void merge_hunit(const Img &a, int64_t u, const U &unite)
{
    const int64_t per = (a.W + HUNIT - 1) / HUNIT;
    const int ty = 1 + (int)(u / per), x0 = (int)(u % per) * HUNIT;
    const int64_t WW = (int64_t)a.nTX * C::NW;  // words per bit-pack row
    const int64_t WP = (int64_t)a.nTX * C::TW;  // ids per tile-edge row
    const int *top = a.edgeRow + (int64_t)(2 * ty) * WP;
    const int *above = a.edgeRow + (int64_t)(2 * ty - 1) * WP;
    auto window = [&](int y) -> uint32_t {
        const uint32_t *row = a.bitpack + CCL_CHK((int64_t)y * WW, (int64_t)a.H * WW, a.status);
        if (x0 == 0)
            return row[0] << 1;  // column -1 is background
        const int xs = x0 - 1, w = xs >> 5, sh = xs & 31;
        uint32_t v = row[w] >> sh;
        if (sh && w + 1 < WW)
            v |= row[w + 1] << (32 - sh);
        return v;
    };
    const uint32_t A = window(ty * C::TH - 1), B = window(ty * C::TH);
    const uint32_t Ash = A << 1, Bsh = B << 1;  // bit j: the column to the left
    const uint32_t sAr = A & ~Ash, sBr = B & ~Bsh;
    const uint32_t cols = ((1u << HUNIT) - 1u) << 1;  // bits 1..HUNIT: columns x0 .. x0 + HUNIT - 1
    uint32_t ev1 = ((C::CONN == 8) ? (sBr & (A | Ash)) : (sBr & A)) & cols;
    uint32_t ev2 = ((C::CONN == 8) ? (sAr & Bsh) : (sAr & B & ~sBr)) & cols & ~ev1;
    int pe = -1, pb = -1;
    while (ev1 | ev2) {
        const uint32_t E = ev1 | ev2;
        const int j = ctz32(E);
        const uint32_t m = 1u << j;
        const bool first = (ev1 & m) != 0u;
        ev1 &= ~m;
        ev2 &= ~m;
        const int x = x0 - 1 + j;
        int xe = x, xb = x;  // the touching B and A pixels
        if (C::CONN == 8) {
            if (first)
                xb = (A & m) ? x : x - 1;
            else
                xe = x - 1;
        }
        const int e = top[CCL_CHK((int64_t)xe, WP, a.status)], bb = above[CCL_CHK((int64_t)xb, WP, a.status)];
#if defined(CCL_DEBUG)
        if (e < 0 || bb < 0) {
            flag_status(a.status, ST_BAD_VALUE);
            continue;
        }
#endif
        if (e == pe && bb == pb)
            continue;
        pe = e;
        pb = bb;
        unite(e, bb);
    }
}

// boundary-merge item i of an image (nh = horizontal_items), joined by `unite`
template <class C, class U> CCL_HD void merge_item(const Img &a, int64_t i, int64_t nh, const U &unite)
{
    if (!C::CLS && i < nh)
        merge_hunit<C>(a, i, unite);
    else
        apply_edge_item<C>(a, load_edge_item<C>(a, i, nh), unite);
}
template <class C> CCL_HD void merge_item(const Img &a, int64_t i, int64_t nh)
{
    merge_item<C>(a, i, nh, UniteGlobal{a});
}

// ---- global phase: flatten (Algorithm 3) and canonical numbering ------------------------
// After the boundary merge every component is a tree over global node ids in which a
// parent always has a smaller id (raster order), and the root is the component's
// raster-first pixel.  Flatten is done by pointer jumping: in each round every node
// follows up to JUMP_HOPS links and points at the farthest node reached, so the reach
// grows geometrically and a path of n nodes needs about log(n)/log(JUMP_HOPS+1) rounds
// (the paper's sequential flatten needs one pass because it visits labels in increasing
// order; that order is not available to parallel threads).
#ifndef CCL_JUMP_HOPS
#define CCL_JUMP_HOPS 32
#endif
constexpr int JUMP_HOPS = CCL_JUMP_HOPS;
constexpr int MAX_ROUNDS = 40;

// One round over the nodes of segment `seg`: every node that is not a root moves its
// parent up to JUMP_HOPS ancestors.  A root is an entry equal to its own id or, once the
// roots are labelled, a negative entry.  Returns true if some node has not reached its
// root; adds the number of roots to *roots.  The parent words of four nodes are loaded
// before any is used (one 16-byte load).
template <class C> CCL_HD bool jump_segment(const Img &a, int64_t seg, int *roots)
{
    const int n = a.nseg[seg];
    const int64_t base = seg * C::ROWCAP;
    bool more = false;
    for (int j0 = 0; j0 < n; j0 += 4) {
        int p4[4];
        ld_g4(&a.P[CCL_CHK(base + j0, a.nP, a.status)], p4);  // a segment's slots are 16-byte aligned
        for (int k = 0; k < 4; k++) {
            const int id = (int)(base + j0 + k);
            const int p = p4[k];
            if (j0 + k >= n)
                continue;
            if (p == id || p < 0) {
                (*roots)++;
                continue;
            }
            int r = (int)CCL_CHK((int64_t)p, a.nP, a.status);
            bool root = false;
            for (int h = 0; h < JUMP_HOPS; h++) {
                const int q = ld_g(&a.P[r]);
                if (q == r || q < 0) {
                    root = true;
                    break;
                }
                r = (int)CCL_CHK((int64_t)q, a.nP, a.status);
            }
            if (r != p)
                st_g(&a.P[id], r);  // only this thread writes P[id] in a round; r is an ancestor
            more |= !root;
        }
    }
    return more;
}

// roots of segments [s0, s1) get -(label): labels continue from `off` in raster order;
// returns the last label given (off if none)
template <class C> CCL_HD int label_roots(const Img &a, int64_t s0, int64_t s1, int off)
{
    for (int64_t seg = s0; seg < s1; seg++) {
        const int n = a.nseg[seg];
        const int64_t base = seg * C::ROWCAP;
        for (int j0 = 0; j0 < n; j0 += 4) {
            int p4[4];
            ld_g4(&a.P[CCL_CHK(base + j0, a.nP, a.status)], p4);
            for (int k = 0; k < 4; k++) {
                const int id = (int)(base + j0 + k);
                if (j0 + k < n && p4[k] == id) {
                    off++;
                    st_g(&a.P[id], -off);
                }
            }
        }
    }
    return off;
}

// contiguous range of segments owned by thread (block b, thread t) for counting/labelling
CCL_HD void seg_range(int64_t nSeg, int nblocks, int nt, int b, int t, int64_t *s0, int64_t *s1)
{
    const int64_t nthreads = (int64_t)nblocks * nt;
    const int64_t per = (nSeg + nthreads - 1) / nthreads;
    const int64_t lo = ((int64_t)b * nt + t) * per;
    *s0 = lo < nSeg ? lo : nSeg;
    *s1 = (lo + per) < nSeg ? (lo + per) : nSeg;
}

// Exclusive scan of one value per thread across a CTA of GNT threads (Hillis-Steele in
// shared memory, double-buffered so that each step reads only the previous step's
// values).  Run as: scan_put; sync; for k < log2(GNT): scan_step(k); sync; then scan_get.
#ifndef CCL_GLOBAL_NT
#define CCL_GLOBAL_NT 1024
#endif
constexpr int GNT = CCL_GLOBAL_NT;
constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }
constexpr int GNT_LOG = ilog2(GNT);
static_assert((1 << GNT_LOG) == GNT, "global CTA size must be a power of two");
template <int N> struct ScanBufT {
    int v[2][N];
};
using ScanBuf = ScanBufT<GNT>;
template <int N> CCL_HD void scan_put(ScanBufT<N> &s, int tid, int x) { s.v[0][tid] = x; }
template <int N> CCL_HD void scan_step(ScanBufT<N> &s, int tid, int k)
{
    const int d = 1 << k;
    const int src = k & 1;
    s.v[src ^ 1][tid] = s.v[src][tid] + (tid >= d ? s.v[src][tid - d] : 0);
}
// inclusive result after ilog2(N) steps lives in buffer ilog2(N) & 1
template <int N> CCL_HD int scan_incl(const ScanBufT<N> &s, int tid) { return s.v[ilog2(N) & 1][tid]; }
// Roots before CTA b: every CTA sums the totals of the CTAs before it itself (after the
// grid barrier that follows the counts), in place of one CTA scanning all totals between
// two barriers.  Returns that sum to every thread; *all receives the grand total.
template <int N> CCL_HD int ctas_before(ScanBufT<N> &s, const int *bsum, int b, int G, int tid, int *all);

// the whole scan: every thread of the CTA (N threads) puts x and gets its inclusive sum
template <int N> CCL_HD int cta_incl_scan(ScanBufT<N> &s, int tid, int x)
{
    scan_put(s, tid, x);
    cta_sync();
    for (int k = 0; k < ilog2(N); k++) {
        scan_step(s, tid, k);
        cta_sync();
    }
    return scan_incl(s, tid);
}

template <int N> CCL_HD int ctas_before(ScanBufT<N> &s, const int *bsum, int b, int G, int tid, int *all)
{
    int x = 0, y = 0;
    for (int i = tid; i < G; i += N) {
        const int v = ld_g(&bsum[i]);
        if (i < b)
            x += v;
        y += v;
    }
    // two sums in one scan: the totals are < 2^31 in all, so pack neither; run twice
    const int before = cta_incl_scan(s, tid, x);
    const int sb = s.v[ilog2(N) & 1][N - 1];
    (void)before;
    cta_sync();
    cta_incl_scan(s, tid, y);
    *all = s.v[ilog2(N) & 1][N - 1];
    cta_sync();
    return sb;
}

// Grid-wide state of the global kernel, in the workspace header.  k_tile_local zeroes it
// before every use (it runs first on the same stream).
struct GridSync {
    unsigned arrive;
    int round_more[MAX_ROUNDS];
    int work_next[2];  // persistent kernel: next tile of its tile phase / of its final phase
    int probe[2];      // persistent kernel: object bytes / bytes in the density probe
};
static_assert(16 + sizeof(GridSync) <= 256, "grid state must fit the 256-byte workspace header");

// ---- kernel bodies (shared by the CUDA kernels and the test emulator) ------------------
// CCL_TICK(k) marks the end of phase k-1 for a phase-timing build (a harness that defines
// CCL_PHASE_TIMING and supplies ccl_phase_tick); it is empty in the library.
#if defined(CCL_PHASE_TIMING) && defined(__CUDACC__)
__device__ void ccl_phase_tick(int kernel, int phase, int tid);
#endif
#if defined(CCL_PHASE_TIMING) && defined(__CUDA_ARCH__)
#define CCL_TICK(kern, k) ccl_phase_tick((kern), (k), tid)
#else
#define CCL_TICK(kern, k) ((void)0)
#endif

// Grid barrier of the cooperative global kernel (all CTAs co-resident).  Each wait is
// capped: after BARRIER_SPIN_CAP polls a CTA records ST_BARRIER and goes on, so a broken
// launch ends with an error status instead of hanging the GPU.
constexpr int BARRIER_SPIN_CAP = 1 << 21;

CCL_HD void grid_sync(GridSync *g, unsigned nblocks, unsigned &epoch, int *status, int tid)
{
#if defined(__CUDA_ARCH__)
    __syncthreads();
    epoch += 1;
    if (tid == 0) {
        __threadfence();
        atomicAdd(&g->arrive, 1u);
        const unsigned target = epoch * nblocks;
        int it = 0;
        while (*reinterpret_cast<volatile unsigned *>(&g->arrive) < target) {
            if (++it > BARRIER_SPIN_CAP) {
                atomicOr(status, ST_BARRIER);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
#else
    (void)g;
    (void)nblocks;
    (void)status;
    (void)tid;
    epoch += 1;
    emu_grid_sync();
#endif
}

// rows a1 + a2 for one tile: bits, strip runs, local Rem union, local roots, run codes,
// global nodes, tile-edge ids
template <class C> CCL_HD void tile_local_body(const Img &a, SmemL<C> &s, int tile, int tid)
{
    using T = Tile<C>;
    const int ty = tile / a.nTX, tx = tile % a.nTX;
    if (tile == 0 && a.gsync) {
        // reset the grid barrier of the global kernel that follows on this stream
        unsigned *g = reinterpret_cast<unsigned *>(a.gsync);
        for (int i = tid; i < (int)(sizeof(GridSync) / 4); i += C::NT)
            g[i] = 0u;
    }
    CCL_TICK(0, 0);
#if CCL_PF_TILE
    T::prefetch_image(a, tile + a.pf_dist, tid);
#endif
    T::load_image(a, s, ty, tx, tid);
    cta_sync();
    CCL_TICK(0, 1);
    T::store_bitpack(a, s, ty, tx, tid);
    T::strip_runs(s, tid);
    cta_sync();
    CCL_TICK(0, 2);
    T::unions(a, s, tid);
    cta_sync();
    CCL_TICK(0, 3);
    T::roots(a, s, tid);
    cta_sync();
    CCL_TICK(0, 4);
    T::mark_roots(a, s, tid);
    cta_sync();
    CCL_TICK(0, 5);
    T::root_prefix(a, s, ty, tx, tid);
    cta_sync();
    CCL_TICK(0, 6);
    T::outputs(a, s, ty, tx, tid);
#if defined(CCL_PHASE_TIMING)
    cta_sync();
    CCL_TICK(0, 7);
#endif
}

// rows a3, a4, a5 (global part) for CTA b of G: boundary merge, pointer-jumping flatten,
// root count, scan and labels.  Roots are final once the merge is done, so they are
// counted during the first jump round and labelled while later rounds (deep trees only)
// keep shortening the other nodes' paths.
template <class C, int NTG = GNT>
CCL_HD void global_body(const Img &a, ScanBufT<NTG> &sb, int &s_flag, int b, int G, int tid)
{
    unsigned epoch = 0;
    GridSync *g = a.gsync;
    const int64_t stride = (int64_t)G * NTG;
    CCL_TICK(1, 0);

    // a3: boundary merge (Algorithm 7's boundary loop with Algorithm 8's union)
    const int64_t nh = horizontal_items<C>(a.nTY, a.W);
    const int64_t nv = (int64_t)(a.nTX - 1) * a.H;
    for (int64_t i = (int64_t)b * NTG + tid; i < nh + nv; i += stride)
        merge_item<C>(a, i, nh);
    grid_sync(g, (unsigned)G, epoch, a.status, tid);
    CCL_TICK(1, 1);

    // a4 + a5: first jump round over this thread's contiguous raster range of segments,
    // counting roots; scan of the counts across the CTA, then across CTAs
    int64_t s0, s1;
    seg_range(a.nSeg, G, NTG, b, tid, &s0, &s1);
    int c = 0;
    bool more = false;
    for (int64_t seg = s0; seg < s1; seg++)
        more |= jump_segment<C>(a, seg, &c);
    if (more)
        flag_status(&g->round_more[0], 1);
    scan_put(sb, tid, c);
    cta_sync();
    for (int k = 0; k < ilog2(NTG); k++) {
        scan_step(sb, tid, k);
        cta_sync();
    }
    const int incl = scan_incl(sb, tid);
    if (tid == NTG - 1)
        st_g(&a.bsum[b], incl);
    grid_sync(g, (unsigned)G, epoch, a.status, tid);
    CCL_TICK(1, 2);
    int total = 0;
    const int before = ctas_before(sb, a.bsum, b, G, tid, &total);
    if (b == G - 1 && tid == 0)
        *a.K = total;
    CCL_TICK(1, 3);
    // root k in raster order receives label k+1 (stored as -(k+1))
    label_roots<C>(a, s0, s1, before + incl - c);

    // further jump rounds while some node has not reached its root
    for (int r = 0; r < MAX_ROUNDS - 1; r++) {
        if (tid == 0)
            s_flag = ld_g(&g->round_more[r]);
        cta_sync();
        const int f = s_flag;
        cta_sync();
        if (!f)
            break;
        bool more_r = false;
        int dummy = 0;
        for (int64_t seg = s0; seg < s1; seg++)
            more_r |= jump_segment<C>(a, seg, &dummy);
        if (more_r)
            flag_status(&g->round_more[r + 1], 1);
        grid_sync(g, (unsigned)G, epoch, a.status, tid);
        if (r == MAX_ROUNDS - 2 && tid == 0 && b == 0 && ld_g(&g->round_more[r + 1]))
            flag_status(a.status, ST_LOOP_CAP);
    }
#if defined(CCL_PHASE_TIMING)
    cta_sync();
    CCL_TICK(1, 4);
#endif
}

// ---- small images: the global phases in one CTA, in shared memory ----------------------
// When an image's segments and nodes fit, one CTA of GNT threads runs rows a3-a5 on a copy
// of the node table in shared memory.  Nodes are numbered densely in raster order (the
// prefix over segments of their root counts); the boundary merge joins them with Rem's
// union on shared words; one find per node flattens; a scan numbers the roots in that
// order (raster order of first pixels, as in global_body); and every node's entry of the
// global table receives -(label).  Each dependent step costs a shared-memory access
// instead of an L2 one, and there is no grid barrier.  An image whose nodes do not fit
// runs global_body in the same CTA (G = 1) on the global table.
constexpr int SMALL_SEG_CAP = 16384;   // segments (image rows x tile columns)
constexpr int SMALL_NODE_CAP = 32768;  // nodes (local components)

struct SmallSmem {
    int pre[SMALL_SEG_CAP + 1];  // nodes before each segment
    int D[SMALL_NODE_CAP];       // dense parents, then -(label)
    ScanBuf sb;
    int flag, n;
};

// Rem's union with splicing on dense ids in shared memory (as rem_unite_g)
CCL_HD void rem_unite_s(int *D, int x, int y, int *st)
{
    int rx = x, ry = y;
    for (int it = 0; it < SMEM_LOOP_CAP; it++) {
        const int px = ld_s(&D[rx]), py = ld_s(&D[ry]);
        if (px == py)
            return;
        if (px > py) {
            if (at_cas(&D[rx], px, py) != px)
                continue;
            if (px == rx)
                return;
            rx = px;
        } else {
            if (at_cas(&D[ry], py, px) != py)
                continue;
            if (py == ry)
                return;
            ry = py;
        }
    }
    flag_status(st, ST_LOOP_CAP);
}

template <class C> struct UniteShared {
    const Img &a;
    int *D;
    const int *pre;
    CCL_HD int dense(int gid) const
    {
        return CCL_CHK(pre[CCL_CHK(gid / C::ROWCAP, (int)a.nSeg, a.status)] + gid % C::ROWCAP, SMALL_NODE_CAP, a.status);
    }
    CCL_HD void operator()(int x, int y) const { rem_unite_s(D, dense(x), dense(y), a.status); }
};

template <class C> CCL_HD void small_global_body(const Img &a, SmallSmem &sm, int tid)
{
    CCL_TICK(1, 0);
    const int nSeg = (int)a.nSeg;
    if (nSeg > SMALL_SEG_CAP) {
        global_body<C>(a, sm.sb, sm.flag, 0, 1, tid);
        return;
    }
    // nodes before each segment
    const int per = (nSeg + GNT - 1) / GNT;
    const int s0 = imin(tid * per, nSeg), s1 = imin(s0 + per, nSeg);
    int c = 0;
    for (int sg = s0; sg < s1; sg++)
        c += a.nseg[sg];
    const int incl = cta_incl_scan(sm.sb, tid, c);
    int run = incl - c;
    for (int sg = s0; sg < s1; sg++) {
        sm.pre[sg] = run;
        run += a.nseg[sg];
    }
    if (tid == GNT - 1) {
        sm.pre[nSeg] = incl;
        sm.n = incl;
    }
    cta_sync();
    const int N = sm.n;
    if (N > SMALL_NODE_CAP) {  // the same decision in every thread
        global_body<C>(a, sm.sb, sm.flag, 0, 1, tid);
        return;
    }
    for (int k = tid; k < N; k += GNT)
        sm.D[k] = k;
    cta_sync();
    // a3: boundary merge
    const int64_t nh = horizontal_items<C>(a.nTY, a.W);
    const int64_t nv = (int64_t)(a.nTX - 1) * a.H;
    const UniteShared<C> unite{a, sm.D, sm.pre};
    for (int64_t i = tid; i < nh + nv; i += GNT)
        merge_item<C>(a, i, nh, unite);
    cta_sync();
    CCL_TICK(1, 1);
    // a4: every node to its root (a node read on the way may already hold its root)
    for (int k = tid; k < N; k += GNT) {
        int r = k;
        for (int it = 0; it < SMEM_LOOP_CAP; it++) {
            const int p = ld_s(&sm.D[r]);
            if (p == r)
                break;
            r = p;
        }
        sm.D[k] = r;
    }
    cta_sync();
    CCL_TICK(1, 2);
    // a5: roots in dense (raster) order get labels 1..K; then every node takes its root's
    const int per2 = (N + GNT - 1) / GNT;
    const int k0 = imin(tid * per2, N), k1 = imin(k0 + per2, N);
    int nr = 0;
    for (int k = k0; k < k1; k++)
        nr += sm.D[k] == k ? 1 : 0;
    const int incl2 = cta_incl_scan(sm.sb, tid, nr);
    int lab = incl2 - nr;
    for (int k = k0; k < k1; k++)
        if (sm.D[k] == k)
            sm.D[k] = -(++lab);
    if (tid == GNT - 1)
        *a.K = incl2;
    cta_sync();
    for (int k = tid; k < N; k += GNT) {
        const int r = sm.D[k];
        if (r >= 0)
            sm.D[k] = sm.D[CCL_CHK(r, N, a.status)];
    }
    cta_sync();
    CCL_TICK(1, 3);
    // every node's entry of the global table, segment by segment
    for (int sg = tid; sg < nSeg; sg += GNT) {
        const int b0 = sm.pre[sg], n = sm.pre[sg + 1] - b0;
        for (int j = 0; j < n; j++)
            a.P[CCL_CHK((int64_t)sg * C::ROWCAP + j, a.nP, a.status)] = sm.D[b0 + j];
    }
#if defined(CCL_PHASE_TIMING)
    cta_sync();
    CCL_TICK(1, 4);
#endif
}

// row a5 (final part) for one tile: label of every strip run, int32 labels
template <class C> CCL_HD void final_body(const Img &a, SmemF<C> &s, int tile, int tid)
{
    using T = Tile<C>;
    const int ty = tile / a.nTX, tx = tile % a.nTX;
    CCL_TICK(2, 0);
#if CCL_PF_FINAL
    T::prefetch_final(a, tile + a.pf_dist, tid);
#endif
    T::load_bitpack(a, s, ty, tx, tid);
    cta_sync();
    CCL_TICK(2, 1);
    T::strip_runs(s, tid);
    cta_sync();
    CCL_TICK(2, 2);
    T::run_labels(a, s, ty, tx, tid);
    cta_sync();
    CCL_TICK(2, 3);
    T::write_labels(a, s, ty, tx, tid);
#if defined(CCL_PHASE_TIMING)
    cta_sync();
    CCL_TICK(2, 4);
#endif
}

// ---- batches: many images, one launch per kernel ---------------------------------------
// Tiles, boundary items and segments of all images are numbered consecutively; prefix
// arrays (n+1 entries) map a number back to its image.  Ranks of global roots run over the
// whole batch; imgBase[i] holds the ranks before image i, and the final pass subtracts it,
// so every image is numbered 1..K_i on its own.  Images with no pixels are left out by the
// host.
struct Batch {
    int n;
    const Img *imgs;           // device array of n per-image descriptors
    const int64_t *tileStart;  // n+1
    const int64_t *itemStart;  // n+1 boundary-merge items
    const int64_t *segStart;   // n+1 segments
    int *imgBase;              // n+1 rank offsets (written by the global kernel)
    GridSync *gsync;
    int *bsum;
    int *status;
    // A batch of one image may carry its descriptor and sizes inline (inl != 0): then
    // imgs and the three prefix arrays are not used (and find_img never reads them for
    // n == 1), so a single-image launch needs no descriptor upload.
    int inl;
    Img one;
    int64_t one_tiles, one_items, one_segs;
    CCL_HD const Img &img(int m) const { return inl ? one : imgs[m]; }
    CCL_HD int64_t tile_start(int k) const { return inl ? (k ? one_tiles : 0) : tileStart[k]; }
    CCL_HD int64_t item_start(int k) const { return inl ? (k ? one_items : 0) : itemStart[k]; }
    CCL_HD int64_t seg_start(int k) const { return inl ? (k ? one_segs : 0) : segStart[k]; }
};

// largest i in [0, n) with start[i] <= x (empty images share their start with the next)
CCL_HD int find_img(const int64_t *start, int n, int64_t x)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// per-CTA copy of the descriptor of the image a tile belongs to
struct TileCtx {
    Img img;
    int tile;
};

template <class C> CCL_HD void batch_tile_local_body(const Batch &B, TileCtx &ctx, SmemL<C> &s, int bid, int tid)
{
    if (tid == 0) {
        const int m = find_img(B.tileStart, B.n, bid);
        ctx.img = B.img(m);
        ctx.tile = (int)(bid - B.tile_start(m));
    }
    if (bid == 0) {
        unsigned *g = reinterpret_cast<unsigned *>(B.gsync);
        for (int i = tid; i < (int)(sizeof(GridSync) / 4); i += C::NT)
            g[i] = 0u;
    }
    cta_sync();
    tile_local_body<C>(ctx.img, s, ctx.tile, tid);
}

template <class C> CCL_HD void batch_final_body(const Batch &B, TileCtx &ctx, SmemF<C> &s, int bid, int tid)
{
    if (tid == 0) {
        const int m = find_img(B.tileStart, B.n, bid);
        ctx.img = B.img(m);
        ctx.tile = (int)(bid - B.tile_start(m));
        ctx.img.label_base = ld_g(&B.imgBase[m]);
        if (ctx.tile == 0 && ctx.img.K)
            *ctx.img.K = ld_g(&B.imgBase[m + 1]) - ctx.img.label_base;
    }
    cta_sync();
    final_body<C>(ctx.img, s, ctx.tile, tid);
}

// The global phases over a batch for CTA b of G CTAs of NTG threads; `epoch` counts the
// grid barriers this CTA has passed (the persistent kernel continues its count).
template <class C, int NTG>
CCL_HD void batch_global_phase(const Batch &B, ScanBufT<NTG> &sb, int &s_flag, int b, int G, int tid,
                               unsigned &epoch)
{
    GridSync *g = B.gsync;
    const int64_t stride = (int64_t)G * NTG;
    const int n = B.n;

    // a3: boundary merge over the items of all images
    const int64_t nitems = B.item_start(n);
    int m = 0;
    for (int64_t i = (int64_t)b * NTG + tid; i < nitems; i += stride) {
        if (i >= B.item_start(m + 1) || i < B.item_start(m))
            m = find_img(B.itemStart, n, i);
        const Img &a = B.img(m);
        merge_item<C>(a, i - B.item_start(m), horizontal_items<C>(a.nTY, a.W));
    }
    grid_sync(g, (unsigned)G, epoch, B.status, tid);

    // a4 + a5: first jump round and root count over a contiguous range of the batch's
    // segments, then the scan across the CTA and across CTAs
    const int64_t nsegs = B.seg_start(n);
    int64_t s0, s1;
    seg_range(nsegs, G, NTG, b, tid, &s0, &s1);
    const int m0 = (s0 < nsegs) ? find_img(B.segStart, n, s0) : n - 1;
    int c = 0;
    bool more = false;
    m = m0;
    for (int64_t seg = s0; seg < s1; seg++) {
        while (seg >= B.seg_start(m + 1))
            m++;
        more |= jump_segment<C>(B.img(m), seg - B.seg_start(m), &c);
    }
    if (more)
        flag_status(&g->round_more[0], 1);
    const int incl = cta_incl_scan(sb, tid, c);
    if (tid == NTG - 1)
        st_g(&B.bsum[b], incl);
    grid_sync(g, (unsigned)G, epoch, B.status, tid);
    int total = 0;
    const int before = ctas_before(sb, B.bsum, b, G, tid, &total);
    if (b == G - 1 && tid == 0)
        st_g(&B.imgBase[n], total);
    // roots get -(batch rank + 1); the thread that meets an image's first segment records
    // the ranks before it
    int run = before + incl - c;
    m = m0;
    for (int64_t seg = s0; seg < s1; seg++) {
        while (seg >= B.seg_start(m + 1))
            m++;
        if (seg == B.seg_start(m))
            st_g(&B.imgBase[m], run);
        const int64_t ls = seg - B.seg_start(m);
        run = label_roots<C>(B.img(m), ls, ls + 1, run);
    }

    for (int r = 0; r < MAX_ROUNDS - 1; r++) {
        if (tid == 0)
            s_flag = ld_g(&g->round_more[r]);
        cta_sync();
        const int f = s_flag;
        cta_sync();
        if (!f)
            break;
        bool more_r = false;
        int dummy = 0;
        m = m0;
        for (int64_t seg = s0; seg < s1; seg++) {
            while (seg >= B.seg_start(m + 1))
                m++;
            more_r |= jump_segment<C>(B.img(m), seg - B.seg_start(m), &dummy);
        }
        if (more_r)
            flag_status(&g->round_more[r + 1], 1);
        grid_sync(g, (unsigned)G, epoch, B.status, tid);
        if (r == MAX_ROUNDS - 2 && tid == 0 && b == 0 && ld_g(&g->round_more[r + 1]))
            flag_status(B.status, ST_LOOP_CAP);
    }
}

template <class C> CCL_HD void batch_global_body(const Batch &B, ScanBuf &sb, int &s_flag, int b, int G, int tid)
{
    unsigned epoch = 0;
    batch_global_phase<C, GNT>(B, sb, s_flag, b, G, tid, epoch);
}

// ---- one persistent launch for a batch (or a single image) -------------------------------
// The phases of k_tile_local, k_global and k_final run back to back in one cooperative grid
// of CTAs of C::NT threads, separated by grid barriers.  Tiles are handed out one at a time
// from a counter (work_next), so CTAs that draw cheap tiles take more of them.  Two tile
// shapes CA and CB can be compiled into one kernel: a density probe at the start (the
// object fraction of a few 16-byte samples of every image) picks the shape for the whole
// launch from the classes the host passes (a row of the tuning table).
template <class A, class B> struct same_t {
    static constexpr bool value = false;
};
template <class A> struct same_t<A, A> {
    static constexpr bool value = true;
};

struct FusedArgs {
    Batch set[2];          // the batch laid out for tile shape CA (0) and CB (1)
    int pick[3];           // shape (0 or 1) per density class: fraction < lo, < hi, >= hi
    int dens_lo, dens_hi;  // class bounds: object fraction in 1/1024
    int probe_samples;     // 16-byte samples per image; 0: no probe, shape pick[0]
};

template <class CA, class CB> union FusedSmemU {
    SmemL<CA> la;
    SmemF<CA> fa;
    SmemL<CB> lb;
    SmemF<CB> fb;
    ScanBufT<CA::NT> sb;
};
template <class CA, class CB> struct FusedSmem {
    FusedSmemU<CA, CB> u;
    TileCtx ctx;
    int next;
    int flag;
    int acc[2];
};

// Object fraction of the batch from probe_samples 16-byte samples per image (sample k of
// an image: row k*H/samples, a column from a multiplicative hash of k); returns the shape
// of its density class.  All CTAs take the same decision after one grid barrier.
template <class CA, class CB>
CCL_HD int fused_probe(const FusedArgs &f, FusedSmem<CA, CB> &sm, int b, int G, int tid, unsigned &epoch)
{
    const Batch &B = f.set[0];
    if (f.probe_samples <= 0)
        return f.pick[0];
    if (tid == 0) {
        sm.acc[0] = 0;
        sm.acc[1] = 0;
    }
    cta_sync();
    const int64_t total = (int64_t)B.n * f.probe_samples;
    int fg = 0, all = 0;
    for (int64_t j = (int64_t)b * CA::NT + tid; j < total; j += (int64_t)G * CA::NT) {
        const int m = (int)(j / f.probe_samples), k = (int)(j % f.probe_samples);
        const Img &a = B.img(m);
        const int y = (int)((int64_t)k * a.H / f.probe_samples);
        const int span = a.W < 16 ? a.W : 16;
        const int x = a.W > 16 ? (int)(((uint32_t)k * 2654435761u) % (uint32_t)(a.W - 15)) : 0;
        const uint8_t *src = a.img + (int64_t)y * a.pitch + x;
        for (int i = 0; i < span; i++)
            fg += (int)src[i] > a.thr ? 1 : 0;
        all += span;
    }
    if (all)
        at_add(&sm.acc[1], all);
    if (fg)
        at_add(&sm.acc[0], fg);
    cta_sync();
    if (tid == 0) {
        at_add(&B.gsync->probe[0], sm.acc[0]);
        at_add(&B.gsync->probe[1], sm.acc[1]);
    }
    grid_sync(B.gsync, (unsigned)G, epoch, B.status, tid);
    const int64_t obj = ld_g(&B.gsync->probe[0]), seen = ld_g(&B.gsync->probe[1]);
    const int64_t d = seen > 0 ? obj * 1024 / seen : 0;
    const int cls = d < f.dens_lo ? 0 : (d < f.dens_hi ? 1 : 2);
    return f.pick[cls];
}

// every phase of the path over batch B laid out for tile shape C
template <class C, class S>
CCL_HD void fused_run(const Batch &B, S &sm, SmemL<C> &sl, SmemF<C> &sf, int b, int G, int tid, unsigned &epoch)
{
    GridSync *g = B.gsync;
    const int ntiles = (int)B.tile_start(B.n);
    // rows a1, a2: tiles from the counter
    for (;;) {
        if (tid == 0) {
            const int t = at_add(&g->work_next[0], 1);
            sm.next = t;
            if (t < ntiles) {
                const int m = find_img(B.tileStart, B.n, t);
                sm.ctx.img = B.img(m);
                sm.ctx.img.gsync = nullptr;  // the grid state is in use: no reset by tile 0
                sm.ctx.tile = (int)(t - B.tile_start(m));
            }
        }
        cta_sync();
        if (sm.next >= ntiles)
            break;
        tile_local_body<C>(sm.ctx.img, sl, sm.ctx.tile, tid);
        cta_sync();
    }
    grid_sync(g, (unsigned)G, epoch, B.status, tid);
    // rows a3, a4, a5 (global part)
    batch_global_phase<C, C::NT>(B, sm.u.sb, sm.flag, b, G, tid, epoch);
    grid_sync(g, (unsigned)G, epoch, B.status, tid);  // the root labels are written
    // row a5 (final part): tiles from the second counter
    for (;;) {
        if (tid == 0) {
            const int t = at_add(&g->work_next[1], 1);
            sm.next = t;
            if (t < ntiles) {
                const int m = find_img(B.tileStart, B.n, t);
                sm.ctx.img = B.img(m);
                sm.ctx.tile = (int)(t - B.tile_start(m));
                sm.ctx.img.label_base = ld_g(&B.imgBase[m]);
                if (sm.ctx.tile == 0 && sm.ctx.img.K)
                    *sm.ctx.img.K = ld_g(&B.imgBase[m + 1]) - sm.ctx.img.label_base;
            }
        }
        cta_sync();
        if (sm.next >= ntiles)
            break;
        final_body<C>(sm.ctx.img, sf, sm.ctx.tile, tid);
        cta_sync();
    }
}

template <class CA, class CB>
CCL_HD void fused_body(const FusedArgs &f, FusedSmem<CA, CB> &sm, int b, int G, int tid)
{
    static_assert(CA::NT == CB::NT, "both tile shapes run with the same CTA size");
    unsigned epoch = 0;
    const int shape = fused_probe<CA, CB>(f, sm, b, G, tid, epoch);
    if constexpr (same_t<CA, CB>::value) {
        (void)shape;
        fused_run<CA>(f.set[0], sm, sm.u.la, sm.u.fa, b, G, tid, epoch);
    } else {
        if (shape == 0)
            fused_run<CA>(f.set[0], sm, sm.u.la, sm.u.fa, b, G, tid, epoch);
        else
            fused_run<CB>(f.set[1], sm, sm.u.lb, sm.u.fb, b, G, tid, epoch);
    }
}

}  // namespace ccl
